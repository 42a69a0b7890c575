"""The batched FP32 GEMM of the FP32 inner solver (SIMT, tcgen05 TF32 and
3xTF32) against an FP64 matrix product of the same FP32 inputs, through the C
ABI.  Shapes span several 128-row tiles with ragged edges, both tile widths
(BN = 64 / 128), all transpose combinations, unaligned leading dimensions
(scalar load path) and two-level k addressing."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# elementwise error bounds relative to (|A| |B|)_ij:
#  SIMT / 3xTF32: FP32 accumulation over k terms plus the 2^-21 split residue
#  TF32: operands rounded to 11 significant bits (2 * 2^-11) plus accumulation
#  BF16 (modes 8, 11): operands rounded to 8 significant bits (2 * 2^-9)
#  BF16 hi/lo split (modes 9, 10): remainders below 2^-18 per operand and the
#  dropped lo*lo product, 4 * 2^-18
def _bound(mode, k):
    u = 2.0 ** -24
    if mode == 1:
        return 2 * 2.0 ** -11 + 2 * k * u
    if mode in (8, 11):
        return 2 * 2.0 ** -9 + 2 * k * u
    if mode in (9, 10):
        return 4 * 2.0 ** -18 + 2 * k * u
    return 2.0 ** -20 + 2 * k * u  # modes 0, 4 (FP32 FMA), 3 and 5-7 (3xTF32)


def _opnd(rng, rows, cols, ld, batch):
    """batch column-major rows x cols FP32 matrices (leading dim ld), packed."""
    buf = np.zeros((batch, cols, ld), dtype=np.float32)
    buf[:, :, :rows] = rng.standard_normal((batch, cols, rows)).astype(np.float32)
    return buf


def _mat(buf, i, rows, cols):
    return buf[i, :, :rows].T.astype(np.float64)  # rows x cols


SHAPES = [
    # m, n, k, pad (ld = rows + pad), batch
    (300, 200, 150, 0, 2),
    (256, 40, 96, 4, 3),      # BN = 64, aligned ld
    (130, 130, 33, 1, 1),     # odd ld: scalar loads; k tail
    (512, 384, 320, 0, 1),
    (200, 17, 160, 0, 5),     # BN = 32 (low-rank factor products, n = rank)
    (1000, 300, 64, 3, 40),   # many tiles per persistent CTA, ragged everywhere
]


@pytest.mark.parametrize("mode", [0, 1, 3, 5, 6, 7, 8, 9, 10, 11])
@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("shape", SHAPES)
def test_gemm_f32(lib, mode, ta, tb, shape):
    """Modes 5-7: 3xTF32 with A, B or both packed (pre-split tiles loaded by
    bulk asynchronous copies); 8 / 9: BF16 operands (kind::f16), rounded or
    split into hi + lo; 10 / 11: those with both operands packed; every
    transpose and the ragged shapes."""
    m, n, k, pad, batch = shape
    rng = np.random.default_rng(m * 7 + n * 3 + k + 100 * ta + 10 * tb + mode)
    ar, ac = (k, m) if ta else (m, k)
    br, bc = (n, k) if tb else (k, n)
    lda, ldb, ldc = ar + pad, br + pad, m + pad
    A = _opnd(rng, ar, ac, lda, batch)
    B = _opnd(rng, br, bc, ldb, batch)
    C0 = _opnd(rng, m, n, ldc, batch)
    alpha, beta = 0.75, -0.5
    dA, dB, dC = (torch.from_numpy(x.ravel().copy()).cuda() for x in (A, B, C0))
    lib.prof_reset()
    lib.prof_enable(True)
    lib.gemm_f32(ta, tb, m, n, k, alpha, dA.data_ptr(), lda, lda * ac, dB.data_ptr(), ldb, ldb * bc, beta,
                 dC.data_ptr(), ldc, ldc * n, batch=batch, mode=mode)
    lib.prof_enable(False)
    tc_launches = lib.prof_query("gemm32tc")[1]
    simt_launches = lib.prof_query("gemm32")[1]
    lib.prof_reset()
    assert (tc_launches > 0) == (mode != 0) and (simt_launches > 0) == (mode == 0)
    Cg = dC.cpu().numpy().reshape(batch, n, ldc)
    for i in range(batch):
        a = _mat(A, i, ar, ac)
        b = _mat(B, i, br, bc)
        opa, opb = (a.T if ta else a), (b.T if tb else b)
        ref = alpha * opa @ opb + beta * _mat(C0, i, m, n)
        scale = abs(alpha) * np.abs(opa) @ np.abs(opb) + abs(beta) * np.abs(_mat(C0, i, m, n))
        got = Cg[i, :, :m].T.astype(np.float64)
        err = np.abs(got - ref)
        assert np.all(err <= _bound(mode, k) * scale + 1e-30), (np.max(err / scale), _bound(mode, k))
        # padding rows of C untouched
        if pad:
            assert np.array_equal(Cg[i, :, m:], C0[i, :, m:])


@pytest.mark.parametrize("mode", [1, 3, 5, 6, 7, 8, 9, 10, 11])
def test_gemm_two_level_k(lib, mode):
    """k runs over panels of kblk columns that sit kstr apart (non-transposed A,
    transposed B), as in the stacked low-rank update of the Sylvester solver."""
    rng = np.random.default_rng(5 + mode)
    m, n, J, kblk = 260, 200, 5, 34
    k = J * kblk
    lda = m + 4
    kstr = lda * (kblk + 3)  # panels with gaps between them
    ldb = n
    kstr_b = kstr  # both operands use the same panel stride
    Abuf = rng.standard_normal(kstr * J).astype(np.float32)
    Bbuf = np.zeros(kstr_b * J + ldb * kblk, dtype=np.float32)
    Bbuf[:] = rng.standard_normal(Bbuf.size).astype(np.float32)

    def col(kk):
        return (kk // kblk) * kstr + (kk % kblk) * lda

    def colb(kk):
        return (kk // kblk) * kstr_b + (kk % kblk) * ldb

    opa = np.stack([Abuf[col(kk):col(kk) + m] for kk in range(k)], axis=1).astype(np.float64)     # m x k
    opb = np.stack([Bbuf[colb(kk):colb(kk) + n] for kk in range(k)], axis=1).astype(np.float64).T  # k x n
    ldc = m
    C0 = np.zeros(ldc * n, dtype=np.float32)
    dA, dB, dC = (torch.from_numpy(x.copy()).cuda() for x in (Abuf, Bbuf, C0))
    # A and B share kblk / kstr in one call: use the B panel stride = A's
    assert kstr_b == kstr
    lib.gemm_f32(0, 1, m, n, k, 1.0, dA.data_ptr(), lda, 0, dB.data_ptr(), ldb, 0, 0.0, dC.data_ptr(), ldc, 0,
                 batch=1, kblk=kblk, kstr=kstr, mode=mode)
    got = dC.cpu().numpy().reshape(n, ldc).T.astype(np.float64)
    ref = opa @ opb
    scale = np.abs(opa) @ np.abs(opb)
    assert np.all(np.abs(got - ref) <= _bound(mode, k) * scale)


def test_gemm_split_beats_tf32(lib):
    """3xTF32 (also with packed operands) must be markedly more accurate than
    plain TF32 on the same data."""
    rng = np.random.default_rng(11)
    m = n = 256
    k = 512
    A = rng.standard_normal((k, m)).astype(np.float32)  # column-major m x k as (k, m) row-major
    B = rng.standard_normal((n, k)).astype(np.float32)
    ref = A.T.astype(np.float64) @ B.T.astype(np.float64)
    errs = {}
    for mode in (1, 3, 7):
        dA, dB = torch.from_numpy(A.ravel().copy()).cuda(), torch.from_numpy(B.ravel().copy()).cuda()
        dC = torch.zeros(m * n, dtype=torch.float32, device="cuda")
        lib.gemm_f32(0, 0, m, n, k, 1.0, dA.data_ptr(), m, 0, dB.data_ptr(), k, 0, 0.0, dC.data_ptr(), m, 0,
                     mode=mode)
        got = dC.cpu().numpy().reshape(n, m).T
        errs[mode] = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert errs[3] < 2e-6 and errs[7] < 2e-6 and errs[1] > 100 * errs[3], errs


def test_gemm_bf16_split_beats_bf16(lib):
    """BF16 operands: the hi/lo split (three products) is about 2^-8 times the
    error of plain BF16 products, packed or not, and plain BF16 sits near its
    8-bit rounding."""
    rng = np.random.default_rng(12)
    m = n = 256
    k = 512
    A = rng.standard_normal((k, m)).astype(np.float32)
    B = rng.standard_normal((n, k)).astype(np.float32)
    ref = A.T.astype(np.float64) @ B.T.astype(np.float64)
    errs = {}
    for mode in (8, 9, 10, 11):
        dA, dB = torch.from_numpy(A.ravel().copy()).cuda(), torch.from_numpy(B.ravel().copy()).cuda()
        dC = torch.zeros(m * n, dtype=torch.float32, device="cuda")
        lib.gemm_f32(0, 0, m, n, k, 1.0, dA.data_ptr(), m, 0, dB.data_ptr(), k, 0, 0.0, dC.data_ptr(), m, 0,
                     mode=mode)
        got = dC.cpu().numpy().reshape(n, m).T
        errs[mode] = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert 5e-4 < errs[8] < 5e-3 and 5e-4 < errs[11] < 5e-3, errs
    assert errs[9] < 3e-5 and errs[10] < 3e-5 and errs[8] > 30 * errs[9], errs


SKINNY_SHAPES = [
    # m, n, k, pad, batch: the skinny kernel's two orientations
    (200, 17, 160, 0, 3),     # n <= 40, ragged long side (two 128-row tiles)
    (640, 34, 300, 2, 2),     # n = 34 (the root-level rational application), k tail
    (130, 40, 64, 1, 1),      # widest skinny n, odd ld (scalar loads)
    (17, 300, 96, 3, 2),      # m <= 64: transposed view (rank x N products)
    (64, 129, 50, 0, 4),      # m at the limit, ragged long side
    (512, 34, 200, 0, 2),     # aligned, n = 34: the cp.async-pipelined kernel (ta = tb = 0)
    (260, 40, 100, 0, 2),     # aligned, ragged m (4-row last tile), k tail inside a chunk
]


@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("shape", SKINNY_SHAPES)
def test_gemm_skinny(lib, ta, tb, shape):
    """The skinny SIMT kernel (mode 4) against an FP64 product, every
    transpose, alpha and beta != 0, padded leading dimensions untouched."""
    m, n, k, pad, batch = shape
    rng = np.random.default_rng(m * 5 + n * 11 + k + 100 * ta + 10 * tb)
    ar, ac = (k, m) if ta else (m, k)
    br, bc = (n, k) if tb else (k, n)
    lda, ldb, ldc = ar + pad, br + pad, m + pad
    A = _opnd(rng, ar, ac, lda, batch)
    B = _opnd(rng, br, bc, ldb, batch)
    C0 = _opnd(rng, m, n, ldc, batch)
    alpha, beta = -1.25, 0.5
    dA, dB, dC = (torch.from_numpy(x.ravel().copy()).cuda() for x in (A, B, C0))
    lib.prof_reset()
    lib.prof_enable(True)
    lib.gemm_f32(ta, tb, m, n, k, alpha, dA.data_ptr(), lda, lda * ac, dB.data_ptr(), ldb, ldb * bc, beta,
                 dC.data_ptr(), ldc, ldc * n, batch=batch, mode=4)
    lib.prof_enable(False)
    assert lib.prof_query("gemm32")[1] > 0 and lib.prof_query("gemm32tc")[1] == 0
    lib.prof_reset()
    Cg = dC.cpu().numpy().reshape(batch, n, ldc)
    for i in range(batch):
        a = _mat(A, i, ar, ac)
        b = _mat(B, i, br, bc)
        opa, opb = (a.T if ta else a), (b.T if tb else b)
        ref = alpha * opa @ opb + beta * _mat(C0, i, m, n)
        scale = abs(alpha) * np.abs(opa) @ np.abs(opb) + abs(beta) * np.abs(_mat(C0, i, m, n))
        got = Cg[i, :, :m].T.astype(np.float64)
        err = np.abs(got - ref)
        assert np.all(err <= _bound(4, k) * scale + 1e-30), np.max(err / scale)
        if pad:
            assert np.array_equal(Cg[i, :, m:], C0[i, :, m:])
