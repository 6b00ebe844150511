"""The C ABI library builds, loads without a GPU and exports every entry
point that include/moto.h declares (no compute call is made here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "moto.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(moto_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for n in ("moto_create", "moto_destroy", "moto_energy_grad", "moto_hvp", "moto_lowest_modes",
              "moto_mmf_step", "moto_descend", "moto_topo_charge", "moto_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2509_26269_gb300 import LIB_PATH, EXPORTED
    lib = ctypes.CDLL(LIB_PATH)
    for n in declared_entry_points():
        assert hasattr(lib, n), n
    assert set(EXPORTED) == set(declared_entry_points())


def test_host_side_calls_without_gpu():
    import paper_2509_26269_gb300 as mo
    p = mo.make_params()
    assert (p.k, p.block, p.krylov_steps, p.lbfgs_mem) == (1, 1, 60, 5)
    assert mo.moto_status_string(mo.MOTO_ERR_NONFINITE).startswith("non-finite")
    # argument validation happens on the host, before any device work
    lib = mo._lib
    h = ctypes.c_void_p()
    bad = mo.make_model(4, 32, J=(1.0,))
    assert lib.moto_create(ctypes.byref(bad), 0, ctypes.byref(p), ctypes.byref(h)) == mo.MOTO_ERR_ARG
    bad = mo.make_model(32, 32, J=(1.0, 0.1, 0.1, 0.1)[:3])
    p2 = mo.make_params(k=9)
    assert lib.moto_create(ctypes.byref(bad), 0, ctypes.byref(p2), ctypes.byref(h)) == mo.MOTO_ERR_ARG
    p3 = mo.make_params(block=8, krylov_steps=13)
    assert lib.moto_create(ctypes.byref(bad), 0, ctypes.byref(p3), ctypes.byref(h)) == mo.MOTO_ERR_ARG
    assert lib.moto_create(ctypes.byref(bad), 7, ctypes.byref(p), ctypes.byref(h)) == mo.MOTO_ERR_ARG


def test_noalloc_rejects_oversized_lattices_on_the_host():
    """The allocation-free energy call holds its partial sums in a fixed array:
    lattices whose stencil blocks would not fit (including sizes whose block
    count overflows 32-bit arithmetic) are refused before any CUDA call."""
    import paper_2509_26269_gb300 as mo
    lib = mo._lib
    fake = ctypes.c_void_p(256)  # never dereferenced: the call must return first
    for L1, L2 in ((8192, 4097), (2147483616, 1056), (1 << 16, 1 << 15), (46341, 46341)):
        big = mo.make_model(L1, L2, J=(1.0,))
        assert lib.moto_energy_grad_noalloc(ctypes.byref(big), 0, fake, None, None, None, None) == mo.MOTO_ERR_ARG
