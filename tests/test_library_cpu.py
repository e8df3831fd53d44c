"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads, exports every entry point
the headers declare, and validates configurations on the host before touching a GPU."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1601_08103_gb300 as lee
from paper_1601_08103_gb300 import build as lb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return lee.load()


def declared_entry_points():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(lee_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_headers_declare_the_boundary():
    names = declared_entry_points()
    for must in ["lee_lbm_create", "lee_lbm_init_fields", "lee_lbm_step", "lee_lbm_moments", "lee_lbm_destroy",
                 "lee_lbm_reduce", "lee_velset_info"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lb.LIB], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_entry_points() if n not in exported]
    assert not missing, missing
    # and the binding's expectations are a subset of the declarations
    assert set(lee.exported_symbols()) <= set(declared_entry_points())


def test_library_is_built_for_sm103a(lib):
    out = subprocess.run(["cuobjdump", "--list-elf", lb.LIB], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_velset_info_matches_paper_tables(lib):
    # the library's own tables, checked against the printed values (tests/golden/velsets.json
    # holds them; here a few spot values suffice since GPU parity checks the rest)
    info = lee.lee_velset_info("D3Q19")
    assert info["q"] == 19 and info["D"] == 3
    shells = {}
    for c, f in zip(info["c"], info["f"]):
        shells.setdefault(sum(abs(v) for v in c), set()).add(round(f, 15))
    assert shells == {0: {round(13 / 40, 15)}, 1: {round(3 / 40, 15)}, 2: {round(3 / 160, 15)}}
    di = lee.lee_velset_info("D3Q7_DI")
    assert di["rho0"] == pytest.approx(1.0) and di["theta0"] == pytest.approx(5 / 21)
    assert di["beta"][1] == pytest.approx(2 / 3) and di["a2"] == pytest.approx(-10.5)
    assert di["c2"] == pytest.approx(147 / 5) and di["gamma"] == pytest.approx(1.4)
    for name in lee.SETS:
        info = lee.lee_velset_info(name)
        assert sum(info["f"]) == pytest.approx(info["rho0"], abs=1e-14)
        vs = set(info["c"])
        assert all(tuple(-v for v in c) in vs for c in vs)


@pytest.mark.parametrize("kw,status", [
    (dict(tau=0.49), lee.LEE_ERR_UNSTABLE_TAU),
    (dict(tau=float("nan")), lee.LEE_ERR_INVALID_ARGUMENT),
    (dict(shape=(0, 4, 1)), lee.LEE_ERR_INVALID_ARGUMENT),
    (dict(shape=(8, 4, 2)), lee.LEE_ERR_INVALID_ARGUMENT),      # 2D set with nz > 1
    (dict(bc="open_sponge", sponge_width=0), lee.LEE_ERR_INVALID_ARGUMENT),
    (dict(bc="open_sponge", sponge_width=4, sponge_strength=1.5), lee.LEE_ERR_INVALID_ARGUMENT),
    (dict(bc="open_sponge", sponge_width=4, shape=(8, 64, 1)), lee.LEE_ERR_INVALID_ARGUMENT),  # frame too wide
    (dict(store_scale=3.0), lee.LEE_ERR_INVALID_ARGUMENT),       # not a power of two
    (dict(set_name="D3Q7", shape=(8, 8, 8), bc="open_learned"), lee.LEE_ERR_UNSUPPORTED),
    (dict(set_name="D3Q19", shape=(8, 8, 8), storage="split16", bc="open_zero"), lee.LEE_ERR_UNSUPPORTED),
    (dict(storage="split16", bc="open_sponge", sponge_width=2), lee.LEE_ERR_UNSUPPORTED),
    (dict(set_name="D1Q3", shape=(64, 1, 1), bc="slab"), lee.LEE_ERR_UNSUPPORTED),   # a slab needs a cut axis
    (dict(bc="open_learned", sponge_width=2, sponge_strength=1.5), lee.LEE_ERR_INVALID_ARGUMENT),  # fallback frame
    (dict(bc="open_learned", sponge_width=4, shape=(16, 8, 1)), lee.LEE_ERR_INVALID_ARGUMENT),     # frame too wide
    (dict(storage="bfp16", bc="slab"), lee.LEE_ERR_UNSUPPORTED),
    (dict(storage="split16", bc="slab"), lee.LEE_ERR_UNSUPPORTED),
    (dict(storage="bfp16", bc="open_learned"), lee.LEE_ERR_UNSUPPORTED),
    (dict(bc="open_sponge", sponge_width=2, storage="bfp16", store_scale=-1.0), lee.LEE_ERR_INVALID_ARGUMENT),
])
def test_create_rejects_bad_configs_on_the_host(lib, kw, status):
    args = dict(set_name="D2Q5", shape=(16, 8, 1), tau=0.6)
    args.update(kw)
    cfg = lee.make_config(args.pop("set_name"), args.pop("shape"), args.pop("tau"), **args)
    h = ctypes.c_void_p()
    assert lib.lee_lbm_create(ctypes.byref(cfg), ctypes.byref(h)) == status
    assert not h.value


def test_null_handle_and_destroy_are_safe(lib):
    assert lib.lee_lbm_destroy(None) == 0
    assert lib.lee_lbm_step(None, 1) == lee.LEE_ERR_INVALID_ARGUMENT
    assert lib.lee_status_string(99) == b"unknown status"


def test_binding_rejects_mixed_host_and_device_buffers():
    a = np.zeros(4)
    assert lee._same_place(a, None, a) == 0


def test_stability_scan_rejects_bad_arguments_on_the_host(lib):
    """Validation happens before any device work, so it runs without a GPU."""
    raw = lee.load()
    assert raw.lee_stability_scan(0, 0.5, 8, 1e-6, None, None, None, None, None) == lee.LEE_ERR_INVALID_ARGUMENT  # rho NULL
    fake = 16  # never dereferenced: every call below fails validation first
    for args in [(0, -1.0, 8, 1e-6), (0, 0.5, 0, 1e-6), (0, 0.5, 8, 0.0), (42, 0.5, 8, 1e-6), (6, 0.5, 300, 1e-6)]:
        assert raw.lee_stability_scan(*args, None, fake, None, None, None) == lee.LEE_ERR_INVALID_ARGUMENT, args


def test_noalloc_binding_rejects_bad_buffers_without_launching(lib):
    """lee_reduce_noalloc's binding checks what the C side cannot (dtype against storage, buffer
    sizes, FP64 output, device placement) and raises before any launch; CPU tensors stand in for
    the caller's buffers, so these checks run without a GPU."""
    import torch

    q, D, cells = 5, 2, 64
    g = torch.zeros((q, cells), dtype=torch.float64)
    out = torch.zeros(D + 4, dtype=torch.float64)
    bad = [
        dict(g=g.float()),                                       # dtype does not match f64 storage
        dict(storage="split16"),                                 # multi-array storage not accepted
        dict(g=torch.zeros((q - 1, cells), dtype=torch.float64)),  # too few elements for q arrays
        dict(pitch=cells + 8),                                   # layout with pitch needs more elements
        dict(cells=0),
        dict(out=torch.zeros(D + 4, dtype=torch.float32)),        # out must be FP64
        dict(out=torch.zeros(D + 3, dtype=torch.float64)),        # out too short
        dict(g=torch.zeros((q, 2 * cells), dtype=torch.float64)[:, ::2]),  # not contiguous
        dict(g=np.zeros((q, cells))),                            # not a tensor
        dict(),                                                  # host tensors: device buffers only
    ]
    for kw in bad:
        args = dict(set_name="D2Q5", storage="f64", g=g, cells=cells, pitch=cells, out=out)
        args.update(kw)
        with pytest.raises(ValueError):
            lee.lee_reduce_noalloc(args["set_name"], args["storage"], args["g"], args["cells"], args["pitch"],
                                   args["out"])


def test_injection_hook_validates_its_argument(lib):
    assert lib.lee_test_inject_cuda_error(-2) == lee.LEE_ERR_INVALID_ARGUMENT
    assert lib.lee_test_inject_cuda_error(-1) == lee.LEE_OK
