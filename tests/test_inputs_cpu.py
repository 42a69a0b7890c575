"""The seeded input generators that serve both the oracle and the CUDA tests:
SplitMix64 against its published reference outputs, and the workload recipes."""
import math

import numpy as np

from paper_1804_05522_gb300 import inputs as I


def test_splitmix64_reference_outputs():
    # outputs of the published reference implementation (Vigna's splitmix64.c)
    r = I.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(5)] == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                                4593380528125082431, 16408922859458223821]
    r = I.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_derived_draws():
    r = I.SplitMix64(7)
    u = np.array([r.uniform() for _ in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    z = I.SplitMix64(8).normal_array((20000,))
    assert abs(z.mean()) < 0.03 and abs(z.var() - 1.0) < 0.05
    k = [I.SplitMix64(9 + i).randint(1, 64) for i in range(2000)]
    assert min(k) == 1 and max(k) == 64


def test_workload_recipes():
    """The shapes and parameters the design notes state for each workload."""
    w = I.WORKLOADS["fd1d_n1024"]()
    op = w.ops[0]
    assert (w.dim, op.N, op.alpha, w.steps, op.shift) == (1, 1024, 1.5, 32, 1.0)
    x = I.grid(1024)
    np.testing.assert_allclose(op.d_plus, math.gamma(1.5) * x ** 1.5)
    np.testing.assert_allclose(op.d_minus, math.gamma(1.5) * (1 - x) ** 1.5)
    np.testing.assert_allclose(w.u0, x ** 2 * (1 - x) ** 2)
    w2 = I.WORKLOADS["fd2d_n4096"]()
    ox, oy = w2.ops
    assert (w2.dim, ox.N, ox.alpha, oy.alpha, w2.steps, ox.leaf, ox.tol) == (2, 4096, 1.5, 1.5, 100, 128, 1e-10)
    assert ox.shift == oy.shift == 0.5
    x = I.grid(4096)
    np.testing.assert_allclose(oy.d_plus, math.gamma(1.5) * (1 + x) ** 1.5)
    np.testing.assert_allclose(oy.d_minus, math.gamma(1.5) * (2 - x) ** 1.5)
    # the paper's 2D source: 100 (sin 10πx cos πy + sin 10t sin πx · y(1-y)), rank 2
    t = 0.37
    F = w2.source(t)
    y = x
    want = 100 * (np.outer(np.sin(10 * np.pi * x), np.cos(np.pi * y))
                  + math.sin(10 * t) * np.outer(np.sin(np.pi * x), y * (1 - y)))
    np.testing.assert_allclose(F, want, rtol=0, atol=1e-12 * np.abs(want).max())
    b = I.batch(count=64, steps=20)
    assert len(b) == 64 and all(wi.dim == (1 if i % 2 == 0 else 2) for i, wi in enumerate(b))
    assert {wi.N for wi in b} <= {512, 1024, 2048, 4096, 8192}
    assert all(1.1 <= op.alpha <= 1.9 for wi in b for op in wi.ops)
