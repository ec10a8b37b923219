"""The allocation-free selection entry point (eptv_select_kth_noalloc).

Some callers cannot allocate device memory -- their device memory is reserved by
another allocator, or they run in a memory-capped service or inside a callback that must
not enter the allocator.  This entry point serves them with working memory compiled into
the library.  Checked here through the C ABI against the handle-based eptv_select_kth,
bit for bit (a selection is exact), on calls back to back: the shared working memory
must not carry anything from one call into the next.  This file is collected last so
that a run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1009_2288_b300 import eptv as E
from paper_1009_2288_b300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def test_noalloc_selection_matches_handle_selection_on_consecutive_calls():
    geo = E.Geometry(I.FanGeometry(3, 5, 2.0, 2.0, 4, 9, 0.02, 0.25, 60.0, 100.0, I.ARC))
    rng = np.random.Generator(np.random.PCG64(2024))
    cases = [(300_001, 270_001), (300_001, 270_001), (4099, 1), (7, 7), (2048, 1024)]
    for n, k in cases:
        vals = rng.uniform(0.0, 1.0, n).astype(np.float32)
        vals[: n // 4] = vals[0]                      # repeated values
        tv = torch.as_tensor(vals, device=DEV)
        a = torch.full((1,), -1.0, device=DEV)
        b = torch.full((1,), -2.0, device=DEV)
        E.eptv_select_kth(geo, tv, k, a)
        E.eptv_select_kth_noalloc(tv, k, b)
        E.eptv_select_kth_noalloc(tv, k, b)           # second call in a row, same answer
        torch.cuda.synchronize()
        assert b.item() == a.item() == float(np.partition(vals, k - 1)[k - 1])


def test_noalloc_selection_rejects_out_of_range_sizes():
    out = torch.empty(1, device=DEV)
    with pytest.raises(E.EptvError) as ei:
        E.eptv_select_kth_noalloc(torch.ones(5, device=DEV), 6, out)
    assert ei.value.code == -1
    with pytest.raises(E.EptvError):
        E.eptv_select_kth_noalloc(torch.ones(5, device=DEV), 0, out)


def test_noalloc_selection_allocates_nothing_and_handles_every_bucket():
    """After a warm-up call the device's free memory does not move across calls.  Values
    spread over all binades (pass-0 buckets across the exponent range), a selected value
    whose low byte is 0xFF (the last bucket of the final 8-bit pass), and a mix of -0.0
    and +0.0 (one key) all select exactly what np.partition selects."""
    rng = np.random.Generator(np.random.PCG64(7))
    n = 200_003
    wide = (rng.uniform(1.0, 2.0, n) * 2.0 ** rng.integers(-126, 127, n)).astype(np.float32)
    x = np.array([0x3F8000FF], dtype=np.uint32).view(np.float32)[0]       # low byte 0xFF
    wide[12345] = x
    k_x = int(np.count_nonzero(wide < x)) + 1
    zeros = np.where(rng.uniform(size=n) < 0.5, np.float32(-0.0), np.float32(0.0)).astype(np.float32)
    zeros[: n // 10] = rng.uniform(0, 1, n // 10).astype(np.float32)
    out = torch.empty(1, device=DEV)
    tw = torch.as_tensor(wide, device=DEV)
    E.eptv_select_kth_noalloc(tw, 1, out)                 # warm-up (looks up the array)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for vals, ks in ((wide, [1, n // 2, k_x, n - 3, n]), (zeros, [1, n // 3, n - n // 10, n])):
        tv = torch.as_tensor(vals, device=DEV)
        for k in ks:
            E.eptv_select_kth_noalloc(tv, k, out)
            torch.cuda.synchronize()
            assert out.item() == float(np.partition(vals, k - 1)[k - 1])
    E.eptv_select_kth_noalloc(tw, k_x, out)
    torch.cuda.synchronize()
    assert out.item() == float(x)
    assert free0 == torch.cuda.mem_get_info()[0]
