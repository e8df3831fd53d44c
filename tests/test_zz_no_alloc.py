"""The allocation-free reduction entry point, lee_reduce_noalloc, against lee_lbm_reduce.

lee_reduce_noalloc serves callers that cannot allocate device memory where they need the global
sums (they run under someone else's allocator or memory budget, or in a phase that must not
allocate) and so cannot create a solver handle.  It keeps its block partials in a fixed device
array inside the library.  This file is collected last on purpose, so that a failure here leaves
every other test already run; it must pass alone in a fresh process as well as after the rest.
"""
import numpy as np
import pytest

import paper_1601_08103_gb300 as lee
from paper_1601_08103_gb300 import inputs

pytestmark = pytest.mark.gpu


def reference_sums(name, storage, g64_dev, scale):
    """The existing entry point: a handle whose state is set to the same populations."""
    info = lee.lee_velset_info(name)
    cells = g64_dev.shape[1]
    with lee.Solver(name, (cells, 1, 1) if info["D"] == 1 else (cells // 4, 4, 1) if info["D"] == 2
                    else (cells // 16, 4, 4), 0.6, storage=storage, store_scale=scale) as sv:
        sv.set_populations(g64_dev)
        out = np.empty(info["D"] + 4)
        sv.reduce(out)
    return out


@pytest.mark.parametrize("name,storage", [("D2Q5", "f64"), ("D3Q19", "f32"), ("D3Q7", "f16"), ("D2Q5_DI", "bf16"),
                                          ("D1Q3", "f32"), ("D1Q3", "bf16")])
def test_noalloc_matches_handle_reduce_on_two_calls_in_a_row(gpu_lib, name, storage):
    """Bit for bit against lee_lbm_reduce on a handle holding the same stored values, on two calls
    in a row with different data (the second call reuses the shared scratch the first one left)."""
    import torch

    info = lee.lee_velset_info(name)
    q, D = info["q"], info["D"]
    cells = 96 * 1024 + 16  # several block tiles and a ragged tail; divisible by 16 for the shapes
    f = torch.tensor(info["f"], dtype=torch.float64, device="cuda")[:, None]
    scale = 1024.0 if storage in ("f16", "bf16") else 1.0
    dtype = {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[storage]
    for call, seed in enumerate((5, 6)):  # two calls in a row, different data
        # the caller's stored populations, in the storage format the library documents (16-bit:
        # S g / f*); the handle gets their exact FP64 values, which it stores back bit for bit
        raw = torch.from_numpy(inputs.random_populations(q, cells, seed, scale=1.0)).cuda()
        stored = raw.to(dtype)
        g64 = stored.double() * (f / scale) if storage in ("f16", "bf16") else stored.double()
        want = reference_sums(name, storage, g64, scale if storage in ("f16", "bf16") else 0.0)
        pitch = cells
        out = torch.full((D + 4,), float("nan"), dtype=torch.float64, device="cuda")
        lee.lee_reduce_noalloc(name, storage, stored, cells, pitch, out, store_scale=scale)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, want), (call, got, want)


def test_noalloc_rejects_bad_arguments(gpu_lib):
    """The C entry point's own checks (called directly, past the binding's checks): sizes beyond
    the fixed scratch, pitch < cells, 16-bit storage without a scale, multi-array storage."""
    import torch

    raw = lee.load()
    g = torch.zeros((5, 64), dtype=torch.float64, device="cuda")
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    d2q5, f64, f16 = lee.SETS["D2Q5"], lee.STORAGE["f64"], lee.STORAGE["f16"]
    for args in [(d2q5, f64, g.data_ptr(), 1 << 31, 1 << 31, 1.0),  # more cells than the scratch serves
                 (d2q5, f64, g.data_ptr(), 64, 32, 1.0),              # pitch < cells
                 (d2q5, f16, g.data_ptr(), 64, 64, 0.0),              # 16-bit storage needs S > 0
                 (d2q5, lee.STORAGE["split16"], g.data_ptr(), 64, 64, 1.0),
                 (d2q5, lee.STORAGE["bfp16"], g.data_ptr(), 64, 64, 1.0),
                 (42, f64, g.data_ptr(), 64, 64, 1.0)]:               # unknown set
        assert raw.lee_reduce_noalloc(*args, out.data_ptr(), st) == lee.LEE_ERR_INVALID_ARGUMENT, args
    # and the binding's own checks raise before any launch
    with pytest.raises(ValueError):
        lee.lee_reduce_noalloc("D2Q5", "f64", g, 1 << 31, 1 << 31, out)
    with pytest.raises(ValueError):
        lee.lee_reduce_noalloc("D2Q5", "f32", g, 64, 64, out)
