"""Host-side check of the integer division the box passes of the denoise
front end use on the GPU: (n + r) / w as the high word of (n + r) * ceil(2^32 / w),
for every box width 3..33 and every sum a pass can produce."""
import numpy as np


def test_multiply_high_division_is_exact():
    for r in range(1, 17):
        w = 2 * r + 1
        mul = ((1 << 32) + w - 1) // w
        top = 65535 * w + r  # the largest (sum + r) of one pass
        for lo in range(0, top + 1, 1 << 22):
            n = np.arange(lo, min(lo + (1 << 22), top + 1), dtype=np.uint64)
            assert np.array_equal((n * np.uint64(mul)) >> np.uint64(32), n // np.uint64(w)), w
