"""The surrogate's tensor-core dense layer (tcgen05) against exact products.

bf16 x bf16 products are exact in FP32 and FP64; the kernel accumulates in
FP32, so against an FP64 sum of the same bf16 values the error is FP32
accumulation rounding: |err| <= K * 2^-24 * sum |a b| per element (a loose
bound; the test uses it directly).  Small-integer inputs are exact.
"""
import numpy as np
import pytest

from paper_2303_14119_gb300 import fk

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fk.load()


def gemm(A, B, N=None):
    """A [M][K], B [N][K] bf16 CUDA tensors -> FP32 [M][N] via the kernel."""
    M, K = A.shape
    N = B.shape[0] if N is None else N
    Cm = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    fk.fk_gemm_bf16_tn(A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), Cm.data_ptr(),
                       Cm.stride(0), M, N, K, err.data_ptr(),
                       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return Cm.cpu()


def test_tiny_integer_product_is_exact():
    g = torch.Generator().manual_seed(1)
    A = torch.randint(-4, 5, (128, 16), generator=g).to(torch.bfloat16)
    B = torch.randint(-4, 5, (16, 16), generator=g).to(torch.bfloat16)
    C = gemm(A.cuda(), B.cuda())
    ref = A.double() @ B.double().T
    assert torch.equal(C.double(), ref)


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (300, 80, 208), (4096, 256, 256),
                                   (256, 16, 4096), (1, 256, 16), (200, 65, 32)])
def test_random_products_within_fp32_accumulation_bound(M, N, K):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = (torch.randn(M, K, generator=g)).to(torch.bfloat16)
    B = (torch.randn(N, K, generator=g)).to(torch.bfloat16)
    C = gemm(A.cuda(), B.cuda())
    ref = A.double() @ B.double().T
    bound = K * 2.0 ** -24 * (A.double().abs() @ B.double().abs().T) + 1e-30
    assert torch.all((C.double() - ref).abs() <= bound)
    # and far tighter than bf16 rounding of the output would be
    assert (C.double() - ref).abs().max() < 1e-3 * ref.abs().max()


def test_strided_operands_and_columns():
    g = torch.Generator().manual_seed(5)
    big_a = torch.randn(150, 96, generator=g).to(torch.bfloat16).cuda()
    big_b = torch.randn(40, 104, generator=g).to(torch.bfloat16).cuda()
    A = big_a[:, :48]   # lda 96, K = 48
    B = big_b[:, :48]   # ldb 104
    C = gemm(A, B)
    ref = A.cpu().double() @ B.cpu().double().T
    assert (C.double() - ref).abs().max() <= 48 * 2.0 ** -24 * (A.cpu().double().abs() @ B.cpu().double().abs().T).max()


def test_bad_shapes_rejected_on_host():
    A = torch.zeros(128, 24, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(16, 24, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(128, 16, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    lib = fk.load()
    import ctypes as Ct
    args = lambda M, N, K, lda=24, ldb=24: (Ct.c_void_p(A.data_ptr()), lda, Ct.c_void_p(B.data_ptr()), ldb,
                                            Ct.c_void_p(C.data_ptr()), 16, M, N, K,
                                            Ct.c_void_p(err.data_ptr()), None)
    assert lib.fk_gemm_bf16_tn(*args(128, 16, 24)) == fk.FK_EINVAL   # K not a multiple of 16
    assert lib.fk_gemm_bf16_tn(*args(128, 300, 16)) == fk.FK_EINVAL  # N > 256
    assert lib.fk_gemm_bf16_tn(*args(128, 16, 16, lda=12)) == fk.FK_EINVAL
    assert lib.fk_gemm_bf16_tn(*args(0, 16, 16)) == fk.FK_EINVAL


# ------------------------------------------------------------ the network
from oracle.mlp_oracle import MLPOracle  # noqa: E402


def init_params(o, seed):
    rng = np.random.default_rng(seed)
    parts = []
    for out_, in_ in o.shapes:
        parts.append(rng.normal(0.0, 1.0 / np.sqrt(in_), out_ * in_))
        parts.append(rng.normal(0.0, 0.05, out_))
    return np.concatenate(parts).astype(np.float32)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


SURROGATE = (6, 256, 3, 65)  # inputs, width, hidden layers, outputs


def test_param_layout_round_trip_and_count():
    o = MLPOracle(*SURROGATE)
    with fk.Mlp(*SURROGATE, max_batch=256) as m:
        assert m.param_count() == o.param_count()
        p = init_params(o, 1)
        m.set_params(p)
        assert np.array_equal(m.get_params(), p)


@pytest.mark.parametrize("n", [1, 130, 300])
def test_forward_matches_oracle(n):
    o = MLPOracle(*SURROGATE)
    p = init_params(o, 2)
    rng = np.random.default_rng(n)
    X = rng.normal(size=(n, 6)).astype(np.float32)
    with fk.Mlp(*SURROGATE, max_batch=512) as m:
        m.set_params(p)
        Y = m.forward(X)
    Yo, _ = o.forward(p.astype(np.float64), X.astype(np.float64), bf16=True)
    assert rel_l2(Y, Yo) <= 1e-3
    # the bf16 rounding is real: without it the oracle is further away
    Y64, _ = o.forward(p.astype(np.float64), X.astype(np.float64), bf16=False)
    assert rel_l2(Y, Y64) > rel_l2(Y, Yo)


def test_forward_in_chunks_equals_one_call():
    o = MLPOracle(*SURROGATE)
    p = init_params(o, 3)
    X = np.random.default_rng(9).normal(size=(333, 6)).astype(np.float32)
    with fk.Mlp(*SURROGATE, max_batch=128) as a, fk.Mlp(*SURROGATE, max_batch=512) as b:
        a.set_params(p)
        b.set_params(p)
        assert np.array_equal(a.forward(X), b.forward(X))


@pytest.mark.parametrize("n", [7, 256, 1000])
def test_gradient_matches_oracle(n):
    o = MLPOracle(*SURROGATE)
    p = init_params(o, 4)
    rng = np.random.default_rng(100 + n)
    X = rng.normal(size=(n, 6)).astype(np.float32)
    T = rng.normal(size=(n, 65)).astype(np.float32)
    w = rng.uniform(0.5, 2.0, 65).astype(np.float32)
    with fk.Mlp(*SURROGATE, max_batch=1024) as m:
        m.set_params(p)
        loss, g = m.loss_grad(X, T, w)
    lo, go = o.loss_grad(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64),
                         w.astype(np.float64), bf16=True)
    assert abs(loss - lo) <= 1e-4 * lo
    pos = 0
    for out_, in_ in o.shapes:
        for size in (out_ * in_, out_):
            seg, ref = g[pos:pos + size], go[pos:pos + size]
            assert rel_l2(seg, ref) <= 5e-3, (pos, size, rel_l2(seg, ref))
            pos += size
    cos = float(np.dot(g, go) / (np.linalg.norm(g) * np.linalg.norm(go)))
    assert cos >= 0.99999


def test_training_reduces_loss_and_is_deterministic():
    o = MLPOracle(6, 64, 2, 5)
    p = init_params(o, 5)
    rng = np.random.default_rng(11)
    X = rng.uniform(-1, 1, size=(2048, 6)).astype(np.float32)
    A = rng.normal(size=(6, 5))
    T = np.sin(X @ A).astype(np.float32)
    runs = []
    for _ in range(2):
        with fk.Mlp(6, 64, 2, 5, max_batch=256) as m:
            m.set_params(p)
            hist = m.train(X, T, batch=128, epochs=60, lr=3e-3, seed=7)
            runs.append((hist, m.get_params()))
    hist = runs[0][0]
    assert hist[-1] < 0.05 * hist[0]
    assert np.array_equal(runs[0][1], runs[1][1]) and np.array_equal(runs[0][0], runs[1][0])
    # the trained network's loss, recomputed by the oracle, agrees
    with fk.Mlp(6, 64, 2, 5, max_batch=2048) as m:
        m.set_params(runs[0][1])
        loss, _ = m.loss_grad(X, T, grad=False)
    lo = o.loss(runs[0][1].astype(np.float64), X.astype(np.float64), T.astype(np.float64), bf16=True)
    assert abs(loss - lo) <= 1e-3 * lo


def test_adam_steps_match_the_fp64_restatement():
    """Two training steps (fk_mlp_train, one batch of one sample per epoch,
    so the batch order is fixed) against Adam (Kingma and Ba 2015) written
    out in FP64 (oracle.mlp_oracle.adam_step), fed the gradients the library
    itself reports at the starting point and after the first step
    (fk_mlp_loss_grad): the parameter changes agree to FP32 rounding."""
    from oracle.mlp_oracle import adam_step
    rng = np.random.default_rng(12)
    dims = (6, 32, 2, 5)
    with fk.Mlp(*dims, max_batch=128) as m:
        p0 = rng.normal(0.0, 0.3, m.param_count()).astype(np.float32)
        x = rng.normal(size=(1, 6)).astype(np.float32)
        t = rng.normal(size=(1, 5)).astype(np.float32)
        lr = 1e-3
        m.set_params(p0)
        _, g0 = m.loss_grad(x, t)
        m.train(x, t, batch=1, epochs=1, lr=lr, seed=3)
        p1 = m.get_params()
        _, g1 = m.loss_grad(x, t)
        m.train(x, t, batch=1, epochs=1, lr=lr, seed=4)
        p2 = m.get_params()
    z = np.zeros(p0.size)
    r1, m1, v1 = adam_step(p0, g0, z, z, 1, lr)
    r2, _, _ = adam_step(p1, g1, m1, v1, 2, lr)
    d1, d1r = p1.astype(np.float64) - p0, r1 - p0
    d2, d2r = p2.astype(np.float64) - p1, r2 - p1.astype(np.float64)
    # the kernel's moments and update are FP32 (relative rounding of a few
    # 1e-7 per operation, bias corrections formed in FP64), and the stored
    # parameter is rounded to its own ulp
    tol = lambda p: 2 * np.spacing(np.abs(p).astype(np.float32)).astype(np.float64) + 1e-5 * lr
    assert np.all(np.abs(d1 - d1r) <= tol(p1)), np.abs(d1 - d1r).max()
    assert np.all(np.abs(d2 - d2r) <= tol(p2)), np.abs(d2 - d2r).max()
    assert np.abs(d1r).max() > 0.5 * lr  # a real step was taken
