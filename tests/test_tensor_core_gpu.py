"""sdp_mixed_gemm: the tensor-core (tcgen05) product of the reduced-precision
Woodbury core formation, against the exact FP64 product.

Rounding the operands from FP64 to FP32 and then to BF16 (unit roundoff 2^-8) or
TF32 (2^-11), u = 2^-8 + 2^-24 or 2^-11 + 2^-24 in all, and accumulating in FP32
bounds every entry by
|C - AB| <= (2u + u^2 + K 2^-24) (|A| |B|)  (each product of rounded operands,
then at most K FP32 roundings of partial sums), so a layout error (a transposed
tile, a wrong swizzle, a skipped K block) shows far above the bound, while a
correct product stays below it.  Sizes are ragged against the 128 x 128 tiles
and the 64-element K blocks.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10973_gb300 import _build, load
    _build.build()
    load()


U = {"bf16": 2.0 ** -8 + 2.0 ** -24, "fp32": 2.0 ** -11 + 2.0 ** -24}


def _mixed(prec, A, B, transA, transB, M, N, K):
    from paper_1703_10973_gb300 import _lib as L
    lib = L.load()
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    Cd = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
    wb = int(lib.sdp_mixed_gemm_work_bytes(M, N, K))
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = lib.sdp_mixed_gemm(L.PREC[prec], M, N, K, C.c_void_p(dA.data_ptr()), A.shape[1], int(transA),
                            C.c_void_p(dB.data_ptr()), B.shape[1], int(transB), C.c_void_p(Cd.data_ptr()), N,
                            C.c_void_p(work.data_ptr()), wb, C.c_void_p(err.data_ptr()),
                            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == L.SDP_OK
    assert int(err.item()) == 0
    return Cd.cpu().numpy()


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
@pytest.mark.parametrize("M,N,K,tA,tB", [(200, 300, 250, False, False), (128, 128, 64, False, False),
                                         (333, 129, 517, True, False), (96, 260, 1000, False, True),
                                         (1, 5, 3, True, True)])
def test_mixed_gemm_within_rounding_bound(prec, M, N, K, tA, tB):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((K, M) if tA else (M, K))
    B = rng.standard_normal((N, K) if tB else (K, N))
    opA = A.T if tA else A
    opB = B.T if tB else B
    got = _mixed(prec, A, B, tA, tB, M, N, K)
    exact = opA @ opB
    u = U[prec]
    bound = (2 * u + u * u + K * 2.0 ** -24) * (np.abs(opA) @ np.abs(opB))
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - exact) <= bound + 1e-300)
    # and it is a reduced-precision product, not an FP64 one
    assert np.abs(got - exact).max() > 1e-12 * np.abs(exact).max()


def test_mixed_gemm_rejects_bad_arguments():
    from paper_1703_10973_gb300 import _lib as L
    lib = L.load()
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = C.c_void_p(x.data_ptr())
    assert lib.sdp_mixed_gemm(L.SDP_FP64, 4, 4, 4, p, 4, 0, p, 4, 0, p, 4, p, 1 << 20, p, None) == L.SDP_ERR_ARG
    assert lib.sdp_mixed_gemm(L.SDP_BF16, 4, 4, 4, p, 4, 0, p, 4, 0, p, 4, p, 8, p, None) == L.SDP_ERR_ARG
    assert lib.sdp_mixed_gemm(L.SDP_BF16, 4, 4, 4, p, 2, 0, p, 4, 0, p, 4, p, 1 << 20, p, None) == L.SDP_ERR_ARG


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_woodbury_core_formed_on_tensor_cores_still_converges(prec):
    """A reduced-precision handle (FP32 or BF16) forms the Algorithm 1 core Z^T (K Z)
    with the tensor-core product in TF32; the core is only a preconditioner, so
    PCG (refined in FP64) still reaches the requested true residual, against the
    oracle's H."""
    import sdp_inputs as si
    from oracle import sdp_oracle as o
    from paper_1703_10973_gb300 import SDPProblem, default_params
    d = si.mc_instance(60, 70, 2, 1500, 14)
    P = o.Problem.from_data(d)
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((d.n, d.n)))
    W = (Q * np.concatenate([rng.uniform(1.0, 3.0, d.n - 2), [150.0, 120.0]])) @ Q.T
    H = o.hessian_entries(P, W)
    r = si.random_vec(d.m, 5)
    out = {}
    for pr in ("fp64", prec):
        with SDPProblem.from_data(d, params=default_params(precond=1, prec=pr)) as p:
            p.set_W(torch.from_numpy(W).cuda().reshape(-1).contiguous())
            p.precond_build()
            z = p.precond_apply(torch.from_numpy(r).cuda()).cpu().numpy()
            y, its, rel, st = p.pcg_solve(torch.from_numpy(r).cuda(), rtol=1e-8, maxit=2000, prec=pr)
            out[pr] = (z, its, rel, y.cpu().numpy())
    z64, z_lp = out["fp64"][0], out[prec][0]
    assert np.linalg.norm(z_lp - z64) > 1e-13 * np.linalg.norm(z64)     # the core differs: tensor cores ran
    y = out[prec][3]
    assert out[prec][2] <= 1e-8
    slack = d.m * np.finfo(float).eps * np.linalg.norm(np.abs(H) @ np.abs(y))
    assert np.linalg.norm(H @ y - r) <= 1.01e-8 * np.linalg.norm(r) + slack
