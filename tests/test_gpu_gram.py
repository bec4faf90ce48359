"""The projected-Gram pass (Eq. THarm_evp; Algorithm 2 steps 6-7) in each of
its arithmetic forms, called through the C ABI (plhr_gram), against the same
products formed in numpy FP64 from the same inputs: element by element, at
ragged row counts (not multiples of the kernels' 32/64-row chunks), for one
block and for a four-block trial basis with a strided block, with and without
the Q family."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plhr():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1408_0042_gb300 as p
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return p


SIGMA = 1068.5711114200


def _blocks(n, ncols, seed, dtype, strided, cs=None):
    """Random blocks shaped like the solver's families: Z of unit-order
    entries, AZ ~ sigma-sized (so that U = AZ - sigma Z has no systematic
    cancellation), and Q = T U for a positive diagonal T (rows scaled by
    weights in [0.5, 1.5] x 1e-3), so that U^T Q is symmetric as in the solver
    (U^T T U); block 2 lives in a wider array (ld > ncols).  cs: the column
    scales the kernels apply (Q is built from U of the scaled columns and
    unscaled again, so that the scaled U^T Q is symmetric)."""
    rng = np.random.default_rng(seed)
    Zs, As = [], []
    for fam_scale, fam in ((1.0, Zs), (SIGMA, As)):
        for b, nc in enumerate(ncols):
            wide = nc + (3 if (strided and b == 2) else 0)
            fam.append((rng.standard_normal((n, wide)) * fam_scale).astype(dtype))
    wts = 1e-3 * rng.uniform(0.5, 1.5, n)[:, None]
    Qs = []
    for Z, A in zip(Zs, As):
        U = A.astype(np.float64) - SIGMA * Z.astype(np.float64)
        Qs.append((wts * U).astype(dtype))
    return Zs, As, Qs


def _ref(Zs, As, Qs, ncols, cs, sigma, f32):
    """FP64 reference from the values the kernels read.  The FP32 forms scale
    and combine in FP32 before the products (the kernels' staging), which the
    reference repeats so that only the products and sums are compared."""
    Z = np.hstack([X[:, :nc] for X, nc in zip(Zs, ncols)]).astype(np.float64)
    A = np.hstack([X[:, :nc] for X, nc in zip(As, ncols)]).astype(np.float64)
    Q = None if Qs is None else np.hstack([X[:, :nc] for X, nc in zip(Qs, ncols)]).astype(np.float64)
    if f32:
        c32 = cs.astype(np.float32)
        z = (Z.astype(np.float32) * c32).astype(np.float64)
        a = (A.astype(np.float32) * c32).astype(np.float64)
        u = a - np.float64(np.float32(sigma)) * z
        q = u if Q is None else (Q.astype(np.float32) * c32).astype(np.float64)
    else:
        z = Z * cs
        u = A * cs - sigma * z
        q = u if Q is None else Q * cs
    return (z, u, q), np.stack([z.T @ z, u.T @ q, q.T @ z])


def _normalised_err(G, ops):
    """max |G - ref| / (|a_i| |b_j|) over the entries (Cauchy-Schwarz scale)."""
    (z, u, q), ref = ops
    nz, nu, nq = (np.linalg.norm(x, axis=0) for x in (z, u, q))
    scale = np.stack([np.outer(nz, nz), np.outer(nu, nq), np.outer(nq, nz)])
    return float(np.max(np.abs(G - ref) / np.maximum(scale, 1e-300)))


# per-form bound on the normalised error: FP64 ~ n u64; double-word: inputs
# rounded once to 2^-48; FP32 forms: the FP32 rounding of the staged inputs
# (2^-24 each) plus FP32 sums of 32 (pipes) or 128 (tensor memory) products
# folded into double-FP32
TOL = {0: 1e-13, 2: 1e-12, 1: 2e-6, 3: 2e-6}


@pytest.mark.parametrize("form", [0, 1, 2, 3])
@pytest.mark.parametrize("n,ncols,strided,with_q", [
    (1, [5], False, True), (63, [20], False, False), (1000, [44], False, True), (4097, [64], False, True),
    (70001, [16, 11, 11, 16], True, True), (70001, [16, 11, 11, 16], True, False), (131072 + 37, [16, 16, 16, 16],
                                                                                    False, True)])
def test_gram_forms_match_fp64_products(plhr, form, n, ncols, strided, with_q):
    f32 = form in (1, 3)
    dt = np.float32 if f32 else np.float64
    Zs, As, Qs = _blocks(n, ncols, 7 + n, dt, strided)
    if not with_q:
        Qs = None
    m = sum(ncols)
    cs = 10.0 ** np.random.default_rng(n).uniform(-1, 1, m)
    td = lambda L: [torch.from_numpy(np.ascontiguousarray(X)).cuda()[:, :nc] for X, nc in zip(L, ncols)]
    G = plhr.gram(form, td(Zs), td(As), None if Qs is None else td(Qs), sigma=SIGMA,
                  colscale=torch.from_numpy(cs).cuda()).cpu().numpy()
    err = _normalised_err(G, _ref(Zs, As, Qs, ncols, cs, SIGMA, f32))
    print("form %d n %d m %d: normalised error %.3e" % (form, n, m, err))
    assert err <= TOL[form]
    assert np.all(np.isfinite(G))


def test_gram_tensor_cores_agree_with_fp32_pipes(plhr):
    """The two FP32 forms compute the same staged products: they agree to the
    FP32 summation level on a 128^3-sized basis column count (m = 64)."""
    n, ncols = 300007, [16, 16, 16, 16]
    Zs, As, Qs = _blocks(n, ncols, 3, np.float32, False)
    cs = np.ones(64)
    td = lambda L: [torch.from_numpy(X).cuda() for X in L]
    g1 = plhr.gram(1, td(Zs), td(As), td(Qs), sigma=SIGMA, colscale=torch.from_numpy(cs).cuda()).cpu().numpy()
    g3 = plhr.gram(3, td(Zs), td(As), td(Qs), sigma=SIGMA, colscale=torch.from_numpy(cs).cuda()).cpu().numpy()
    ops = _ref(Zs, As, Qs, ncols, cs, SIGMA, True)
    assert _normalised_err(g1, ops) <= TOL[1] and _normalised_err(g3, ops) <= TOL[3]
    # Z^T Z symmetric in both
    assert np.abs(g3[0] - g3[0].T).max() <= 1e-6 * np.abs(np.diag(g3[0])).max()


def test_gram_rejects_bad_arguments(plhr):
    Z = torch.zeros((10, 65), dtype=torch.float64, device="cuda")
    with pytest.raises(plhr.PlhrError):
        plhr.gram(0, Z, Z)                                  # m > 64
    Z = torch.zeros((10, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(plhr.PlhrError):
        plhr.gram(7, Z, Z)                                  # unknown form
