"""The allocation-free projected eigensolve (plhr_tharm_extract_noalloc).

It is for callers that cannot allocate device memory when they call it (an
application whose allocator owns the device, a fixed memory budget, a host
callback).  It must give what plhr_tharm_extract gives on the same inputs,
also on consecutive calls that share its built-in scratch array, and reject a
basis larger than that array serves.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from oracle import operators as oops

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1408_0042_gb300 as p
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    L = p.load_library()
    fn = L.plhr_tharm_extract_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p] * 11
    return p, L


def _problem(seed, nv, nrest):
    rng = np.random.default_rng(seed)
    A = oops.laplacian_dirichlet((20, 20), 1 / 21).toarray()
    n = A.shape[0]
    M = rng.standard_normal((n, n))
    T = np.linalg.inv(A + 50.0 * np.eye(n))
    T = 0.5 * (T + T.T) + 1e-4 * (M @ M.T) / n
    sigma = 300.0
    m = nv + nrest
    Z = rng.standard_normal((n, m)) * 10.0 ** rng.uniform(-3, 1, m)[None, :]
    cs = 10.0 ** rng.uniform(-1, 1, m)
    Zs = Z * cs[None, :]
    U = A @ Zs - sigma * Zs
    Q = T @ U
    return Zs.T @ Zs, U.T @ Q, Q.T @ Zs, cs, nv


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _noalloc(L, Gzz, Guq, Gqz, cs, kp, nv):
    m = Gzz.shape[0]
    outs = {"Cp": torch.zeros((m, kp), dtype=torch.float64, device="cuda"),
            "Cvv": torch.zeros((nv, kp), dtype=torch.float64, device="cuda"),
            "tags": torch.zeros(kp, dtype=torch.int32, device="cuda"),
            "partner": torch.zeros(kp, dtype=torch.int32, device="cuda"),
            "xi": torch.zeros(2 * kp, dtype=torch.float64, device="cuda"),
            "status": torch.zeros(3, dtype=torch.int32, device="cuda")}
    ins = [_dev(Gzz), _dev(Guq), _dev(Gqz), _dev(cs)]
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in ins + list(outs.values())]
    st = L.plhr_tharm_extract_noalloc(m, kp, nv, *ptrs, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == 0, L.plhr_last_error().decode()
    res = {k: v.cpu().numpy() for k, v in outs.items()}
    res["units"] = int(res["status"][2])
    return res


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(lib):
    p, L = lib
    # two different problems in a row: the second call reuses the scratch the
    # first one left behind
    for seed, nv, nrest in [(11, 16, 48), (12, 5, 15), (13, 11, 33)]:
        Gzz, Guq, Gqz, cs, nv = _problem(seed, nv, nrest)
        ref = p.tharm_extract(_dev(Gzz), _dev(Guq), _dev(Gqz), _dev(cs), nv, nv)
        got = _noalloc(L, Gzz, Guq, Gqz, cs, nv, nv)
        assert ref["status"] == 0 and got["status"][0] == 0
        assert got["status"][1] == ref["kept"] and got["units"] == ref["units"]
        assert np.array_equal(got["tags"], ref["tags"])
        assert np.array_equal(got["partner"], ref["partner"])
        np.testing.assert_allclose(got["xi"][: 2 * ref["units"]], ref["xi"].ravel(), rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(got["Cp"], ref["Cp"], rtol=1e-12, atol=1e-14 * np.abs(ref["Cp"]).max())
        np.testing.assert_allclose(got["Cvv"], ref["Cvv"], rtol=1e-12, atol=1e-14 * np.abs(ref["Cvv"]).max())


def test_noalloc_call_leaves_device_free_memory_unchanged(lib):
    """After its first call on the device, a call with the caller's buffers in
    place allocates nothing: the device's free memory is the same before and
    after it (both read after a synchronise)."""
    p, L = lib
    Gzz, Guq, Gqz, cs, nv = _problem(14, 16, 48)
    m, kp = Gzz.shape[0], nv
    ins = [_dev(Gzz), _dev(Guq), _dev(Gqz), _dev(cs)]
    outs = [torch.zeros((m, kp), dtype=torch.float64, device="cuda"),
            torch.zeros((nv, kp), dtype=torch.float64, device="cuda"),
            torch.zeros(kp, dtype=torch.int32, device="cuda"), torch.zeros(kp, dtype=torch.int32, device="cuda"),
            torch.zeros(2 * kp, dtype=torch.float64, device="cuda"), torch.zeros(3, dtype=torch.int32, device="cuda")]
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in ins + outs]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.plhr_tharm_extract_noalloc(m, kp, nv, *ptrs, stream) == 0     # set-up call
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert L.plhr_tharm_extract_noalloc(m, kp, nv, *ptrs, stream) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert int(outs[5][0].item()) == 0


def test_noalloc_rejects_basis_beyond_its_scratch(lib):
    p, L = lib
    buf = torch.zeros(65 * 65, dtype=torch.float64, device="cuda")
    ib = torch.zeros(64, dtype=torch.int32, device="cuda")
    ptr = ctypes.c_void_p(buf.data_ptr())
    iptr = ctypes.c_void_p(ib.data_ptr())
    st = L.plhr_tharm_extract_noalloc(65, 4, 4, ptr, ptr, ptr, ptr, ptr, ptr, iptr, iptr, ptr, iptr, None)
    assert st == p.PLHR_EINVAL
    assert "exceeds the maximum" in L.plhr_last_error().decode()
