"""CPU oracle for the SLRME dual-layer lossless RGBE coder.

Test infrastructure only: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.
"""
