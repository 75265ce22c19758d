"""The C ABI without a GPU: the library builds, loads and exports every entry
point that include/hd.h declares; argument validation happens on the host;
without a device the product path fails loudly instead of falling back."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hd.h")


@pytest.fixture(scope="module")
def hdlib():
    import paper_1211_1645_gb300 as hd
    return hd, hd.load()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hd_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_paper_calls():
    syms = declared_symbols()
    for name in ("hd_init", "hd_sweep", "hd_pressure", "hd_psi6", "hd_positions"):
        assert name in syms


def test_library_exports_every_declared_symbol(hdlib):
    hd, lib = hdlib
    out = subprocess.run(["nm", "-D", "--defined-only", hd.build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    for s in declared_symbols():
        assert hasattr(lib, s)


def test_status_strings_and_defaults(hdlib):
    hd, lib = hdlib
    from paper_1211_1645_gb300 import hd as b
    assert b.status_string(0) == "ok"
    assert "argument" in b.status_string(1)
    o = b.hd_default_opts()
    assert (o.precision, o.lattice, o.hist_bins, o.hist_dr, o.cell_min) == (0, 0, 50, 1e-3, 2.0)
    assert (o.strips, o.replica_branches, o.threads_per_cell) == (0, 0, 1)


@pytest.mark.parametrize("N,eta,sigma,delta,kw", [
    (1, 0.7, 1.0, 0.1, {}),                       # fewer than two disks
    (256, 0.0, 1.0, 0.1, {}),                     # eta <= 0
    (256, 0.79, 1.0, 0.1, {}),                    # square lattice would overlap
    (256, 0.7, 1.0, -0.1, {}),                    # negative step
    (256, 0.7, 1.0, 3.0, {}),                     # step beyond the cell side
    (256, 0.7, 1.0, 1e-300, {}),                  # step below 2^-900 sigma (and not 0)
    (9, 0.7, 1.0, 0.1, {}),                       # fewer than 4 cells per side
    (256, 0.7, 1.0, 0.1, {"cell_min": 1.5}),      # cells narrower than a diameter
    (256, 0.7, 1.0, 0.1, {"hist_bins": 10000}),   # too many bins for the fit
    (256, 0.7, 1.0, 0.1, {"hist_bins": 4}),       # too few bins for a quartic
    (256, 0.7, 1.0, 0.1, {"block_threads": 100}),  # not a warp multiple
    (256, 0.7, 1.0, 0.1, {"threads_per_cell": 3}),  # not 1, 2, 4 or 8 lanes
    (256, 0.7, 1.0, 0.1, {"threads_per_cell": 8}),  # 128 cells x 8 lanes > 512 threads
    (256, 0.7, 1.0, 0.1, {"threads_per_cell": 2, "sweep_kernel": "tma"}),  # groups only in the split pass
    (256, 0.7, 1.0, 0.1, {"cell_min": [1.9]}),     # a per-replica cell side below a diameter
    (256, 0.7, 1.0, 0.1, {"strips": -1}),          # strips: 0 automatic, 1 none, 2 .. 64
    (256, 0.7, 1.0, 0.1, {"strips": 65}),
    (256, 0.7, 1.0, 0.1, {"strips": 9}),           # m = 16: eight bands, fewer than nine strips
    (256, 0.7, 1.0, 0.1, {"strips": 2, "sweep_kernel": "tma"}),  # strips only on the split kernels
    (256, 0.7, 1.0, 0.1, {"strips": 2, "threads_per_cell": 2}),  # ... with one thread per cell
    (256, 0.7, 1.0, 0.1, {"replica_branches": 2}),  # 0 automatic or 1 off
])
def test_invalid_arguments_rejected_on_host(hdlib, N, eta, sigma, delta, kw):
    hd, lib = hdlib
    from paper_1211_1645_gb300 import hd as b
    opts = b.make_opts(**kw)
    h = ctypes.c_void_p()
    st = lib.hd_init(ctypes.byref(h), N, eta, sigma, delta, 1, ctypes.byref(opts))
    assert st == b.HD_ERR_ARG
    assert not h.value


def test_batch_replica_count_bounds(hdlib):
    """1 <= R <= 65535 (the per-block replica tables hold 16-bit indices);
    the count is checked before any per-replica array is read."""
    hd, lib = hdlib
    from paper_1211_1645_gb300 import hd as b
    one_n = (ctypes.c_int64 * 1)(256)
    one_d = (ctypes.c_double * 1)(0.7)
    one_s = (ctypes.c_uint64 * 1)(1)
    h = ctypes.c_void_p()
    for R in (0, 65536):
        st = lib.hd_batch_init(ctypes.byref(h), ctypes.c_int32(R), one_n, one_d, ctypes.c_double(1.0), one_d, one_s,
                               None)
        assert st == b.HD_ERR_ARG and not h.value


def test_strips_need_a_single_replica(hdlib):
    """Strips split one replica's grid; a batch takes replica branches instead."""
    hd, lib = hdlib
    from paper_1211_1645_gb300 import hd as b
    n = (ctypes.c_int64 * 2)(256, 256)
    d = (ctypes.c_double * 2)(0.7, 0.7)
    dl = (ctypes.c_double * 2)(0.1, 0.1)
    sd = (ctypes.c_uint64 * 2)(1, 2)
    h = ctypes.c_void_p()
    opts = b.make_opts(strips=2)
    st = lib.hd_batch_init(ctypes.byref(h), ctypes.c_int32(2), n, d, ctypes.c_double(1.0), dl, sd, ctypes.byref(opts))
    assert st == b.HD_ERR_ARG and not h.value


def test_null_context_calls(hdlib):
    hd, lib = hdlib
    from paper_1211_1645_gb300 import hd as b
    assert lib.hd_sweep(None, 1) == b.HD_ERR_ARG
    assert lib.hd_positions(None, None) == b.HD_ERR_ARG
    assert lib.hd_destroy(None) == b.HD_OK
    assert lib.hd_replicas(None) == 0
    assert lib.hd_psi6_acf(None, 3, None) == b.HD_ERR_ARG
    assert lib.hd_psi6_tau(None, 1, 2, None) == b.HD_ERR_ARG
    assert lib.hd_psi6_field(None, 4, None) == b.HD_ERR_ARG
    assert lib.hd_structure_factor(None, 1, None, None) == b.HD_ERR_ARG
    assert lib.hd_positional_q0(None, 1, None, None) == b.HD_ERR_ARG
    assert lib.hd_positional_field(None, None, 4, None) == b.HD_ERR_ARG
    assert lib.hd_positional_corr(None, None, 4, 0.5, None) == b.HD_ERR_ARG


def test_no_cpu_fallback_without_gpu(hdlib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    hd, lib = hdlib
    from paper_1211_1645_gb300 import hd as b
    with pytest.raises(b.HDError) as e:
        b.hd_init(256, 0.7, 1.0, 0.1, 1)
    assert e.value.status == b.HD_ERR_CUDA


def comment_of_each_declaration():
    """Map each declared hd_* call to the comment that documents it: the
    nearest block comment before its declaration that starts a line (comments
    trailing code on a line, such as field notes, are not documentation of a
    call).  One block may document a group of calls declared under it."""
    text = open(HEADER).read()
    out = {}
    last = ""
    for m in re.finditer(r"(?m)^[ \t]*(/\*.*?\*/)|/\*.*?\*/|\b(hd_[a-z0-9_]+)\s*\(", text, flags=re.S):
        if m.group(1):
            last = m.group(1)
        elif m.group(2):
            out.setdefault(m.group(2), last)
    return out


def test_every_call_cites_its_passage():
    """Each exported call's comment names the section, equation or table of
    the paper that defines it, or states that the paper has no counterpart."""
    cites = re.compile(r"Sec\.|Eqs?\.|Table|no counterpart")
    docs = comment_of_each_declaration()
    missing = [s for s in declared_symbols() if not cites.search(docs.get(s, ""))]
    assert not missing, missing


def test_noalloc_rejects_misaligned_pointers_on_host(hdlib):
    """The allocation-free Psi_6 mean reads doubles: a pointer that is not
    8-byte aligned is rejected before any device work (no GPU needed)."""
    hd, lib = hdlib
    from paper_1211_1645_gb300 import hd as b
    V = ctypes.c_void_p
    assert lib.hd_psi6_mean_noalloc(V(0x10004), ctypes.c_int64(16), V(0x20000), None) == b.HD_ERR_ARG
    assert lib.hd_psi6_mean_noalloc(V(0x10000), ctypes.c_int64(16), V(0x20004), None) == b.HD_ERR_ARG
    assert lib.hd_psi6_mean_noalloc(None, ctypes.c_int64(16), V(0x20000), None) == b.HD_ERR_ARG
    assert lib.hd_psi6_mean_noalloc(V(0x10000), ctypes.c_int64(0), V(0x20000), None) == b.HD_ERR_ARG
