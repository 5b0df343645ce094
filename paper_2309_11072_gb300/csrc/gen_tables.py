"""Writes tables.inc: the codec's constant tables as literals.

Run from the repository root after changing a definition:
    python paper_2309_11072_gb300/csrc/gen_tables.py

Tables (all built in float64 and rounded once):
  kLog2Lut[i]   = round(65536 * log2(2048 + i)),        i = 0..2047
  kGammaBits[k] = float32 bits of ((k - 0.5) / 255)^2.2,  k = 1..255 (k = 0: 0.0)
  kKrBits[r]    = float32 bits of 0.18 * 2^(-r/16),        r = 0..15
  kWrBits[r]    = float32 bits of 1800 * 2^(-r/16),        r = 0..15
  kGammaStart[b] = #{k in 1..255 : gamma[k] <= start of bucket b}, where
                  bucket b = 256 (e - 107) + m holds the float32 values with
                  biased exponent e in 107..126 and top 8 mantissa bits m
                  (v in [2^-20, 1)); no bucket holds more than one threshold,
                  so the display code of v is start + (v >= gamma[start + 1]).
  kGammaCode[i] = the display code as one word per coarser bucket, i = 0 ..
                  2561: bucket i - 1 (biased exponent e in 107..126 and top 7
                  mantissa bits) for i = 1 .. 2560, i = 0 for v < 2^-20 and
                  i = 2561 for v >= 1; no such bucket holds more than one
                  threshold either.  Entry i belongs to the float bits whose
                  high half is 0x357F + i (bits(v) clamped to 0x357F0000 ..
                  0x3F800000 first), and its word is, mod 2^32,
                  ((start - 0x357F - i) << 16) + 0x10000 - t, with start the
                  count of thresholds below the bucket and t the low 16 bits of
                  the one threshold inside it, or 0x10000 (no 16-bit value
                  reaches it) when there is none; since
                  (bits(v) & 0xFFFF) + 0x10000 - t < 0x20000, the code of v is
                  (bits(v) + word) >> 16 = start + ((bits(v) & 0xFFFF) >= t).
The literals live in the library's device and host code, so no table has to
be built or copied at run time.

jpeg_tables.inc holds the Huffman code lengths of the base layer's entropy
coding (T.81 Annex K.3: Tables K.3 and K.5, luminance; K.4 and K.6,
chrominance, as kJpegDcLenC and kJpegAcLenC):
  kJpegDcLen[c]  = code length of DC category c (0..11; 0 for 12..15)
  kJpegAcLen[rs] = code length of AC symbol rs = (run << 4) | size: the
                   table's symbols with codes shorter than 16 bits take the
                   lengths listed below, every other symbol with size 1..10
                   (and ZRL, EOB when listed) a 16-bit code, all others 0.
"""
import math
import os
import struct


def f32_bits(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", x))[0]


def main():
    lut = [round(65536.0 * math.log2(2048 + i)) for i in range(2048)]
    gamma = [0] + [f32_bits(((k - 0.5) / 255.0) ** 2.2) for k in range(1, 256)]
    kr = [f32_bits(0.18 * 2.0 ** (-r / 16.0)) for r in range(16)]
    # buckets of [2^-20, 1) by exponent and top 8 mantissa bits; thresholds as
    # bit patterns (positive floats order like their bits)
    assert gamma[1] > (107 << 23) and gamma[255] < (127 << 23)
    start = []
    for b in range(20 * 256):
        lo = (107 << 23) + (b << 15)
        hi = lo + (1 << 15)
        k = sum(1 for t in gamma[1:] if t <= lo)
        inside = [t for t in gamma[1:] if lo < t < hi]
        assert len(inside) <= 1 and (k == 255 or k + 2 > 255 or gamma[k + 2] >= hi), b
        start.append(k)
    wr = [f32_bits(1800.0 * 2.0 ** (-r / 16.0)) for r in range(16)]
    def word(i, start, t):
        return (((start - 0x357F - i) << 16) + 0x10000 - t) & 0xFFFFFFFF

    code = [word(0, 0, 0x10000)]
    for b in range(20 * 128):
        lo = (107 << 23) + (b << 16)
        hi = lo + (1 << 16)
        assert lo >> 16 == 0x357F + b + 1
        k = sum(1 for t in gamma[1:] if t < lo)
        inside = [t for t in gamma[1:] if lo <= t < hi]
        assert len(inside) <= 1, b
        code.append(word(b + 1, k, (inside[0] & 0xFFFF) if inside else 0x10000))
    assert (127 << 23) >> 16 == 0x357F + len(code)
    code.append(word(len(code), 255, 0x10000))
    def arr(ctype, name, vals, fmt, per_line):
        lines = []
        for i in range(0, len(vals), per_line):
            lines.append("    " + ", ".join(fmt(v) for v in vals[i:i + per_line]) + ",")
        return f"SLRME_TABLE {ctype} {name}[{len(vals)}] = {{\n" + "\n".join(lines) + "\n};\n"

    out = ["// Generated by gen_tables.py -- do not edit.  Constant tables of the codec.",
           "// Include after defining SLRME_TABLE (storage class / qualifiers).", ""]
    out.append(arr("int32_t", "kLog2Lut", lut, str, 12))
    out.append(arr("uint32_t", "kGammaBits", gamma, lambda v: f"0x{v:08x}u", 8))
    out.append(arr("uint32_t", "kKrBits", kr, lambda v: f"0x{v:08x}u", 8))
    out.append(arr("uint32_t", "kWrBits", wr, lambda v: f"0x{v:08x}u", 8))
    out.append(arr("uint8_t", "kGammaStart", start, str, 24))
    out.append(arr("uint32_t", "kGammaCode", code, lambda v: f"0x{v:08x}u", 8))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tables.inc")
    with open(path, "w") as fh:
        fh.write("\n".join(out))

    # Table K.3: DC luminance, code lengths by category 0..11
    dc = [2, 3, 3, 3, 3, 3, 4, 5, 6, 7, 8, 9] + [0] * 4
    # Table K.5: AC luminance, the symbols of codes shorter than 16 bits by length
    short = {2: [0x01, 0x02], 3: [0x03], 4: [0x00, 0x04, 0x11], 5: [0x05, 0x12, 0x21], 6: [0x31, 0x41],
             7: [0x06, 0x13, 0x51, 0x61], 8: [0x07, 0x22, 0x71], 9: [0x14, 0x32, 0x81, 0x91, 0xa1],
             10: [0x08, 0x23, 0x42, 0xb1, 0xc1], 11: [0x15, 0x52, 0xd1, 0xf0], 12: [0x24, 0x33, 0x62, 0x72],
             15: [0x82]}
    ac = [16 if 1 <= (rs & 15) <= 10 else 0 for rs in range(256)]
    for length, syms in short.items():
        for rs in syms:
            ac[rs] = length
    valid = {0x00, 0xF0} | {(r << 4) | z for r in range(16) for z in range(1, 11)}
    assert {rs for rs in range(256) if ac[rs]} == valid
    assert sum(2.0 ** -ac[rs] for rs in valid) == 1.0 - 2.0 ** -16
    assert sum(2.0 ** -l for l in dc[:12]) == 1.0 - 2.0 ** -9
    # Table K.4: DC chrominance; Table K.6: AC chrominance (codes shorter than 16 bits by length)
    dc_c = [2, 2, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11] + [0] * 4
    short_c = {2: [0x00, 0x01], 3: [0x02], 4: [0x03, 0x11], 5: [0x04, 0x05, 0x21, 0x31],
               6: [0x06, 0x12, 0x41, 0x51], 7: [0x07, 0x61, 0x71], 8: [0x13, 0x22, 0x32, 0x81],
               9: [0x08, 0x14, 0x42, 0x91, 0xa1, 0xb1, 0xc1], 10: [0x09, 0x23, 0x33, 0x52, 0xf0],
               11: [0x15, 0x62, 0x72, 0xd1], 12: [0x0a, 0x16, 0x24, 0x34], 14: [0xe1], 15: [0x25, 0xf1]}
    ac_c = [16 if 1 <= (rs & 15) <= 10 else 0 for rs in range(256)]
    for length, syms in short_c.items():
        for rs in syms:
            ac_c[rs] = length
    assert {rs for rs in range(256) if ac_c[rs]} == valid
    assert sum(2.0 ** -ac_c[rs] for rs in valid) == 1.0 - 2.0 ** -16
    assert sum(2.0 ** -l for l in dc_c[:12]) == 1.0 - 2.0 ** -11
    out = ["// Generated by gen_tables.py -- do not edit.  Huffman code lengths of JPEG's",
           "// typical tables (T.81 Annex K.3: luminance K.3, K.5; chrominance K.4, K.6).",
           "// Include after defining SLRME_TABLE.", ""]
    out.append(arr("uint8_t", "kJpegDcLen", dc, str, 16))
    out.append(arr("uint8_t", "kJpegAcLen", ac, str, 16))
    out.append(arr("uint8_t", "kJpegDcLenC", dc_c, str, 16))
    out.append(arr("uint8_t", "kJpegAcLenC", ac_c, str, 16))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "jpeg_tables.inc")
    with open(path, "w") as fh:
        fh.write("\n".join(out))


if __name__ == "__main__":
    main()
