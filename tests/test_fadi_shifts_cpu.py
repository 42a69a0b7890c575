"""Host logic of the factored-ADI shift selection (§3.3) through the C ABI, on
the CPU: the Gershgorin intervals of the D&C blocks against dense spectra and
row sums, and the Zolotarev shifts against the rational function they define,
evaluated independently on fine grids, and against the Beckermann–Townsend
upper bound on the Zolotarev number."""
import math

import numpy as np
import pytest

from oracle import fde_oracle as O
from paper_1804_05522_gb300 import binding
from paper_1804_05522_gb300 import inputs as I


@pytest.fixture(scope="module")
def lib():
    from paper_1804_05522_gb300 import build

    build.build()  # incremental: recompiles only what changed since the last build
    return binding.load()


def _blocks(N, leaf):
    return [rng for lvl in O.hodlr_tree(N, leaf) for rng in lvl]


@pytest.mark.parametrize("side", [0, 1])
def test_block_interval_row_sums_and_spectrum(lib, side):
    """lam_lo is the smallest row sum of the block, lam_hi the largest
    a_ii + Σ_j |a_ij| (both from the dense operator), and every eigenvalue's
    real part lies between them, for every node of the tree."""
    w = I.fd2d(N=150, alpha=(1.3, 1.8), steps=20, leaf=16)
    op = w.ops[side]
    A = O.fd_operator(op)
    p = lib.op_params(op)
    for lo, hi in _blocks(op.N, 16):
        B = A[lo:hi, lo:hi]
        lam_lo, lam_hi = lib.fde_block_interval(p, lo, hi)
        rows = B.sum(axis=1)
        gersh = np.diag(B) + (np.abs(B).sum(axis=1) - np.abs(np.diag(B)))
        scale = np.abs(B).max()
        assert lam_lo == pytest.approx(rows.min(), rel=0, abs=1e-12 * scale), (lo, hi)
        assert lam_hi == pytest.approx(gersh.max(), rel=0, abs=1e-12 * scale), (lo, hi)
        ev = np.linalg.eigvals(B).real
        assert lam_lo > 0 and ev.min() >= lam_lo * (1 - 1e-12) and ev.max() <= lam_hi * (1 + 1e-12)


def _ratio_fine(al, be, a, b, c, d, G=20001):
    z = np.concatenate([a * (b / a) ** np.linspace(0, 1, G), np.linspace(a, b, G)])
    x = np.concatenate([c * (d / c) ** np.linspace(0, 1, G), np.linspace(c, d, G)])
    rz = np.prod(np.abs((z[:, None] - al) / (z[:, None] - be)), axis=1)
    rw = np.prod(np.abs((-x[:, None] - al) / (-x[:, None] - be)), axis=1)
    return rz.max() / rw.min()


def _bt_bound(J, a, b, c, d):
    """Beckermann–Townsend: Z_J(E, F) <= 4 exp(-π² J / log(16 γ)), γ the cross
    ratio of E = [a, b] and F = [-d, -c]."""
    gamma = (d + a) * (c + b) / ((d + b) * (c + a))
    return 4.0 * math.exp(-math.pi ** 2 * J / math.log(16.0 * gamma))


INTERVALS = [(1.0, 10.0, 1.0, 10.0), (0.5, 3e3, 0.7, 5e3), (2e-3, 40.0, 1e-2, 900.0), (1.0, 1e6, 3.0, 2e5)]


@pytest.mark.parametrize("a,b,c,d", INTERVALS)
@pytest.mark.parametrize("target", [1e-5, 1e-13])
def test_fadi_shifts_zolotarev(lib, a, b, c, d, target):
    al, be, ratio = lib.fde_fadi_shifts(a, b, c, d, target)
    J = len(al)
    assert 1 <= J < 64
    # zeros in E, poles in F
    assert np.all((al >= a * (1 - 1e-12)) & (al <= b * (1 + 1e-12)))
    assert np.all((be <= -c * (1 - 1e-12)) & (be >= -d * (1 + 1e-12)))
    # the reported ratio is what the shifts give on a 50x finer grid (within 1 %),
    # so the target is met
    fine = _ratio_fine(al, be, a, b, c, d)
    assert fine <= ratio * 1.01 and fine >= ratio * (1 - 1e-9)
    assert fine <= target * 1.01
    # optimal shifts reach the Zolotarev number, which is below the
    # Beckermann–Townsend bound
    assert fine <= _bt_bound(J, a, b, c, d) * (1 + 1e-6)
    # J is the smallest count that meets the target
    if J > 1:
        al1, _, r1 = lib.fde_fadi_shifts(a, b, c, d, target, jmax=J - 1)
        assert len(al1) == J - 1 and r1 > target


def test_fadi_shifts_geometric_rate(lib):
    """The ratio falls geometrically in J at the rate the bound predicts
    (each extra shift gains at least the factor exp(-π²/log(16γ)) / 2)."""
    a, b, c, d = 1.0, 1e4, 1.0, 1e4
    prev = None
    rate = math.exp(-math.pi ** 2 / math.log(16.0 * ((d + a) * (c + b) / ((d + b) * (c + a)))))
    for J in range(1, 9):
        al, be, r = lib.fde_fadi_shifts(a, b, c, d, 1e-300 + 1e-16, jmax=J)
        assert len(al) == J
        if prev is not None:
            assert r <= prev * rate * 2.0, (J, r, prev)
        prev = r


@pytest.mark.parametrize("args", [(0.0, 1.0, 1.0, 2.0, 1e-5, 8), (2.0, 1.0, 1.0, 2.0, 1e-5, 8),
                                  (1.0, 2.0, 1.0, 1.0, 1e-5, 8), (1.0, 2.0, 1.0, 2.0, 1.0, 8),
                                  (1.0, 2.0, 1.0, 2.0, 1e-5, 0), (1.0, 2.0, 1.0, 2.0, 1e-5, 65)])
def test_fadi_shifts_rejects_bad_arguments(lib, args):
    with pytest.raises(binding.FdeError) as e:
        lib.fde_fadi_shifts(*args[:5], jmax=args[5])
    assert e.value.status == binding.FDE_ERR_ARG


def test_block_interval_rejects_bad_ranges(lib):
    op = I.fd1d(N=64).ops[0]
    p = lib.op_params(op)
    for lo, hi in [(-1, 4), (4, 4), (10, 65), (5, 2)]:
        with pytest.raises(binding.FdeError) as e:
            lib.fde_block_interval(p, lo, hi)
        assert e.value.status == binding.FDE_ERR_ARG


def test_fadi_shifts_random_intervals(lib):
    """Random interval pairs spanning 1 to 8 decades: the shifts meet the
    target on a fine grid, stay below the Beckermann–Townsend bound, and J is
    minimal."""
    rng = np.random.default_rng(3305)
    for _ in range(60):
        a = 10.0 ** rng.uniform(-3, 1)
        b = a * 10.0 ** rng.uniform(0.5, 8)
        c = 10.0 ** rng.uniform(-3, 1)
        d = c * 10.0 ** rng.uniform(0.5, 8)
        target = 10.0 ** rng.uniform(-13, -3)
        al, be, ratio = lib.fde_fadi_shifts(a, b, c, d, target)
        J = len(al)
        fine = _ratio_fine(al, be, a, b, c, d, G=4001)
        assert fine <= target * 1.02 and fine <= ratio * 1.01, (a, b, c, d, target, J)
        assert fine <= _bt_bound(J, a, b, c, d) * (1 + 1e-6), (a, b, c, d, J)
        if J > 1:
            assert lib.fde_fadi_shifts(a, b, c, d, target, jmax=J - 1)[2] > target
