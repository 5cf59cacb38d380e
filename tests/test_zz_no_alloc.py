"""tm_apply_D_noalloc: the allocation-free variant of tm_apply_D.

It exists for callers that may not allocate device memory during a call (a fixed memory
budget held by a caching allocator, a hard per-process limit, or a latency-critical loop
where cudaMalloc/cudaFree would synchronise the device).  Its work buffers come from one
static device array shared by all calls.  This file is collected last so that a failure
here does not hide the other tests in a run that stops at the first failure.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_0905_3331_gb300 import Lattice, inputs, tm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fn():
    lib = tm.load()
    f = lib.tm_apply_D_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                  ctypes.c_int, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return lib, f


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("T,L", [(4, 4), (32, 16)])
def test_noalloc_matches_apply_D_twice(T, L):
    lib, fn = _fn()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    U = inputs.random_gauge(T, L, 0.5, 1)
    lat = Lattice(T, L, 0.1632, 0.004)
    lat.set_gauge(torch.from_numpy(U).to(dev))
    nrhs = 2
    src = torch.from_numpy(inputs.gaussian_spinor(T, L, 5, shape_prefix=(nrhs,))).to(dev)
    stream = torch.cuda.current_stream().cuda_stream
    for dagger in (0, 1):
        ref = torch.empty_like(src)
        lat.apply_D(ref, src, flavour=1, dagger=bool(dagger), nrhs=nrhs)
        outs = [torch.full_like(src, float("nan")) for _ in range(2)]
        for k in range(2):  # two calls in a row share (and reuse) the static scratch
            st = fn(lat._h, outs[k].data_ptr(), src.data_ptr(), 1, dagger, nrhs, stream)
            assert st == 0, lib.tm_last_error()
        torch.cuda.synchronize()
        for out in outs:
            assert _rel(out, ref) < 1e-13
    # after the set-up call, a further call leaves the device's free memory unchanged
    out = torch.empty_like(src)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    assert fn(lat._h, out.data_ptr(), src.data_ptr(), -1, 0, nrhs, stream) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    lat.close()


def test_noalloc_first_call_on_a_fresh_lattice_matches_the_oracle():
    """The entry point as the first operator call on a freshly created lattice (no tm_apply_D
    before it, so no lattice work space exists), for M and M^dag with two right-hand sides:
    compared with the CPU oracle's M directly (M^dag = gamma5 M(-mu) gamma5), and the
    device's free memory is the same before and after the call."""
    lib, fn = _fn()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream().cuda_stream
    # the per-device set-up (the scratch array's address) happens on some earlier call; make
    # one on another lattice so that this test also holds in a fresh process
    warm = Lattice(4, 4, 0.16, 0.01)
    warm.set_gauge(torch.from_numpy(inputs.unit_gauge(4, 4)).to(dev))
    wx = torch.zeros(4 ** 4 * 12, dtype=torch.complex128, device=dev)
    wy = torch.empty_like(wx)
    assert fn(warm._h, wy.data_ptr(), wx.data_ptr(), 1, 0, 1, stream) == 0, lib.tm_last_error()
    torch.cuda.synchronize()
    warm.close()
    T, L, kappa, mu = 8, 6, 0.1615, 0.003
    U = inputs.random_gauge(T, L, 0.6, 3)
    nrhs = 2
    src_np = inputs.gaussian_spinor(T, L, 9, shape_prefix=(nrhs,))
    lat = Lattice(T, L, kappa, mu)
    lat.set_gauge(torch.from_numpy(U).to(dev))
    src = torch.from_numpy(src_np).to(dev)
    olat = oracle.Lattice.cubic(T, L)
    g5 = np.diag([1.0, 1.0, -1.0, -1.0])
    for dagger in (0, 1):
        out = torch.full_like(src, float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        st = fn(lat._h, out.data_ptr(), src.data_ptr(), 1, dagger, nrhs, stream)
        torch.cuda.synchronize()
        assert st == 0, lib.tm_last_error()
        assert torch.cuda.mem_get_info(dev)[0] == free0
        got = out.cpu().numpy()
        for r in range(nrhs):
            if dagger:
                v = np.einsum("ab,...bc->...ac", g5, src_np[r])
                ref = np.einsum("ab,...bc->...ac", g5, oracle.apply_M(olat, U, v, kappa, -mu))
            else:
                ref = oracle.apply_M(olat, U, src_np[r], kappa, mu)
            assert np.linalg.norm(got[r] - ref) / np.linalg.norm(ref) < 1e-13
    lat.close()


def test_noalloc_rejects_what_it_cannot_do():
    lib, fn = _fn()
    dev = torch.device("cuda:0")
    big = Lattice(48, 24, 0.16, 0.01)  # V = 663552 > 174762: over the scratch limit
    x = torch.zeros(8, dtype=torch.complex128, device=dev)
    y = torch.zeros(8, dtype=torch.complex128, device=dev)
    assert fn(big._h, x.data_ptr(), y.data_ptr(), 1, 0, 1, 0) == 1  # TM_ERR_ARG
    assert b"limit" in lib.tm_last_error()
    big.close()
    lat = Lattice(4, 4, 0.16, 0.01)
    lat.set_gauge(inputs.unit_gauge(4, 4))
    host_in = np.zeros((4, 4, 4, 4, 4, 3), dtype=np.complex128)
    host_out = np.zeros_like(host_in)
    assert fn(lat._h, host_out.ctypes.data, host_in.ctypes.data, 1, 0, 1, 0) == 1
    assert b"device memory" in lib.tm_last_error()
    if torch.cuda.device_count() > 1:  # memory of another GPU is rejected, not read remotely
        other = torch.zeros(4 ** 4 * 12, dtype=torch.complex128, device="cuda:1")
        mine = torch.zeros_like(other, device=dev)
        assert fn(lat._h, mine.data_ptr(), other.data_ptr(), 1, 0, 1, 0) == 1
        assert b"lattice's device" in lib.tm_last_error()
        assert fn(lat._h, other.data_ptr(), mine.data_ptr(), 1, 0, 1, 0) == 1
    lat.close()
