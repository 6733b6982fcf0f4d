"""CPU checks of the blocked mixed leaf's memory plan, read from the library's own layout code
(the host-only test hook tsqr_internal_wy_layout, which calls the kernel's layout, tensor-memory
and Z tile-set functions).  For every width up to 112 columns and every chunk height that fits
one GB300 CTA's shared memory (227 KB opt-in, less the 1 KB the planner keeps free) and an SM's
512 tensor-memory columns, every panel's partial Z tiles fit their slots (an overflow of those
slots once wrote past the end of shared memory at 65-72 columns); and AUTO's height, the tallest
that fits, is the one the GPU tests expect."""
import ctypes

import pytest

OPTIN = 232448  # bytes of shared memory a GB300 CTA may opt in to
HEIGHTS = (1024, 768, 640, 512, 384, 256)  # tallest first, as the planner tries them


@pytest.fixture(scope="module")
def layout():
    from paper_1002_4250_gb300 import _build
    _build.build()
    import paper_1002_4250_gb300 as T
    fn = T._load().tsqr_internal_wy_layout
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
    fn.restype = ctypes.c_int

    def call(n, h):
        out = (ctypes.c_int64 * 4)()
        assert fn(n, h, out) == 0
        return tuple(out)  # smem bytes, tensor-memory columns, most partial tiles, slots
    return call


def _fits(smem, tmem):
    return smem + 1024 <= OPTIN and tmem <= 512


def test_partial_tiles_fit_at_every_height_that_fits(layout):
    for n in range(1, 113):
        fitting = 0
        for h in HEIGHTS:
            smem, tmem, most, slots = layout(n, h)
            if _fits(smem, tmem):
                fitting += 1
                assert most <= slots, (n, h, most, slots)
        assert fitting >= 1, n  # every width up to 112 has a chunk height


def test_auto_heights(layout):
    def auto_h(n):
        return next(h for h in HEIGHTS if _fits(*layout(n, h)[:2]))
    for n in range(1, 113):
        expect = (1024 if n <= 32 else 768 if n <= 48 else 640 if n <= 64 else 512 if n <= 80
                  else 384 if n <= 96 else 256)
        assert auto_h(n) == expect, n


def test_the_slots_are_used_to_the_full(layout):
    """At 112 columns the first panel's 12 n-tiles take 4 tile sets (2 row groups): 24 partial
    tiles, exactly the slots.  At 72 columns the first panel's 7 n-tiles take 4 sets too (14
    tiles, where 2 sets would need 28) and the third panel's 3 n-tiles one set of 8 row groups:
    24 again."""
    assert layout(112, 256)[2:] == (24, 24)
    assert layout(72, 512)[2:] == (24, 24)
