"""GPU test of hd_psi6_mean_noalloc: the global Psi_6 entry point for callers
that cannot allocate device memory when they call it (inside a stream
capture, under a framework that owns all allocations, or in a loop where an
allocation could stall).  It must give the same Psi_6 as hd_psi6 on the same
field, bit for bit (both sum exactly and round once), on consecutive calls
that reuse its fixed scratch array.  This file is named to be collected
last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _call(lib, field, N, out, stream):
    return lib.hd_psi6_mean_noalloc(ctypes.c_void_p(field.data_ptr()), ctypes.c_int64(N),
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def test_noalloc_psi6_matches_library_psi6():
    torch = pytest.importorskip("torch")
    import paper_1211_1645_gb300 as hd
    lib = hd.load()
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    # two calls in a row: one block of partial sums, then 74 blocks; the
    # second field is read from an odd double offset (8-byte aligned only)
    for N, eta, seed, form in [(4096, 0.70, 3, "fixed"), (300000, 0.71, 4, "fp64")]:
        sysg = hd.HardDisks(N, eta, 0.1, seed, precision=form)
        sysg.sweep(20)
        glob, loc = sysg.psi6()
        flat = torch.from_numpy(np.stack([loc.real, loc.imag], 1).ravel().copy())
        off = 0 if N == 4096 else 1
        buf = torch.zeros(2 * N + off, dtype=torch.float64)
        buf[off:] = flat
        field = buf.to("cuda")[off:]
        torch.cuda.synchronize()
        assert _call(lib, field, N, out, stream) == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert complex(got[0], got[1]) == glob[0]
        sysg.close()


def test_noalloc_rejects_out_of_range_sizes():
    torch = pytest.importorskip("torch")
    import paper_1211_1645_gb300 as hd
    from paper_1211_1645_gb300.hd import HD_ERR_ARG
    lib = hd.load()
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert _call(lib, buf, 0, out, 0) == HD_ERR_ARG
    assert _call(lib, buf, 4096 * 4096 + 1, out, 0) == HD_ERR_ARG
