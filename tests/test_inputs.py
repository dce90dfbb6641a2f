"""The seeded workload generator: determinism, recipe shapes and statistics."""
import math

import numpy as np
import pytest

from paper_2203_10148_gb300 import inputs


def test_splitmix64_published_vector():
    """SplitMix64 with state 0 (key 0): the first outputs of the published
    generator are 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F."""
    s = inputs.SeededStream(0)
    got = [int(v) for v in s.u64(3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_stream_is_deterministic_and_counter_based():
    a = inputs.SeededStream(1234).uniform(10)
    s = inputs.SeededStream(1234)
    b = np.concatenate([s.uniform(4), s.uniform(6)])
    np.testing.assert_array_equal(a, b)
    assert np.all((a >= 0) & (a < 1))


def test_normal_statistics():
    z = inputs.SeededStream(7).normal(200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_heat1d_recipe():
    w = inputs.heat1d()
    assert (w.M, w.N, w.fine, w.coarse) == (63, 16, ("ie", 100), ("ie", 1))
    x = np.arange(1, 64) / 64.0
    noise = w.y0[0] - (np.sin(math.pi * x) + 0.5 * np.sin(3 * math.pi * x))
    assert 2e-4 < noise.std() < 3e-3


def test_heat2d_recipe():
    w = inputs.heat2d(n=32, N=8)
    assert w.y0.shape == (1, 1024) and w.fine == ("rk4", 50)
    assert w.y0.min() >= 0.0 and w.y0.max() > 0.05
    w2 = inputs.heat2d(n=32, N=8, batch=3)
    np.testing.assert_array_equal(w2.y0[0], w.y0[0])
    assert not np.array_equal(w2.y0[1], w2.y0[0])


def test_advdiff_recipe_velocity():
    w = inputs.advdiff2d(n=64, N=4)
    speed = np.sqrt(w.vx ** 2 + w.vy ** 2)
    # scaled to unit maximum speed, then sampled as FP32 values (each
    # component rounded once: at most 2^-24 relative)
    assert abs(speed.max() - 1.0) < 2.0 ** -23
    assert np.array_equal(w.vx.astype(np.float32).astype(np.float64), w.vx)
    assert np.array_equal(w.vy.astype(np.float32).astype(np.float64), w.vy)
    # v = curl psi is divergence free: the central-difference divergence is
    # O(h^2) small relative to |grad v|
    n = 64
    vx, vy = w.vx.reshape(n, n), w.vy.reshape(n, n)
    div = (np.roll(vx, -1, 1) - np.roll(vx, 1, 1) + np.roll(vy, -1, 0) - np.roll(vy, 1, 0)) * n / 2
    grad = np.abs(np.roll(vx, -1, 1) - np.roll(vx, 1, 1)).max() * n / 2
    assert np.abs(div).max() < 0.05 * grad


def test_advdiff_step_rule_matches_reading():
    # dt = min(0.4 h, 0.2 h^2/nu) with h = 1/512, nu = 5e-3, dT = 0.5/256 gives 13 steps
    assert inputs.advdiff2d_rk4_steps(512, 5e-3, 0.5 / 256) == 13


def test_dense_recipe_is_contractive():
    w = inputs.dense(M=64, N=4)
    sym = 0.5 * (w.A + w.A.T)
    assert np.linalg.eigvalsh(sym).max() <= -0.1 + 1e-12


def test_serving_stream():
    reqs = inputs.serving_stream(count=64)
    assert all(b.arrival > a.arrival for a, b in zip(reqs, reqs[1:]))
    kinds = {w.kind for w in reqs}
    assert kinds == {"heat1d", "heat2d"}
    for w in reqs:
        assert 16 <= w.N <= 1024
        if w.kind == "heat1d":
            assert 63 <= w.M <= 4095 and w.fine == ("ie", 100)
        else:
            assert 32 <= w.nx <= 256 and w.fine[1] >= 50
    again = inputs.serving_stream(count=64)
    np.testing.assert_array_equal(again[17].y0, reqs[17].y0)


@pytest.mark.parametrize("pde", ["diffusion", "diffusion_reaction", "advection_diffusion_reaction"])
def test_paper_pde_operator_is_consistent(pde):
    """The finite-difference operator of the Sec. 4 test problems applied to
    f = cos(pi x) cos(pi y) (zero on the boundary of the centred unit square)
    matches mu Lap f - u . grad f - r f to O(h^2), u = (-y, x)."""
    mu, r, adv = inputs.PAPER_PDES[pde]
    errs = []
    for n in (19, 39):
        w = inputs.paper_pde(pde, n=n, N=4)
        h = 1.0 / (n + 1)
        xs = -0.5 + h * np.arange(1, n + 1)
        X, Y = np.meshgrid(xs, xs, indexing="xy")
        f = np.cos(np.pi * X) * np.cos(np.pi * Y)
        fx = -np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)
        fy = -np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y)
        Lf = -2 * np.pi ** 2 * mu * f - r * f
        if adv:
            Lf = Lf - ((-Y) * fx + X * fy)
        got = (w.A @ f.ravel()).reshape(n, n)
        errs.append(np.abs(got - Lf).max() / np.abs(Lf).max())
    assert errs[0] < 5e-3 and errs[1] < errs[0] / 3.0     # second order


def test_paper_pde_shapes_and_steps():
    w = inputs.paper_pde("advection_diffusion_reaction", n=49, N=16)
    assert w.M == 2401 and w.A.shape == (2401, 2401)
    assert w.fine == ("ie", 400) and w.coarse == ("ie", 1) and w.T == 6.4
    assert abs(w.y0.max() - 1.0) < 1e-12


def test_fem_p1_matrices_exact_properties():
    """P1 assembly on the uniform triangulation cut along one diagonal has
    closed forms: K is the 5-point stencil (4 on the diagonal, -1 for the
    four axis neighbours, 0 for the diagonal ones), Mm has h^2/2 on the
    diagonal and h^2/12 for each of the six edge neighbours (axis and the
    (+1, +1) / (-1, -1) diagonal), and the convection matrix of the
    divergence-free u = (-y, x) is skew-symmetric once Dirichlet nodes are
    removed."""
    n = 9
    Mm, K, C = inputs.fem_p1_matrices(n, True)
    h = 1.0 / (n + 1)
    Kx = np.zeros((n * n, n * n))
    Mx = np.zeros((n * n, n * n))
    for j in range(n):
        for i in range(n):
            r = j * n + i
            Kx[r, r] = 4.0
            Mx[r, r] = h * h / 2.0
            for di, dj, k, m in ((1, 0, -1, 1), (-1, 0, -1, 1), (0, 1, -1, 1), (0, -1, -1, 1),
                                 (1, 1, 0, 1), (-1, -1, 0, 1)):
                if 0 <= i + di < n and 0 <= j + dj < n:
                    Kx[r, (j + dj) * n + i + di] = k
                    Mx[r, (j + dj) * n + i + di] = m * h * h / 12.0
    np.testing.assert_allclose(K, Kx, atol=1e-13)
    np.testing.assert_allclose(Mm, Mx, atol=1e-16)
    assert np.abs(C + C.T).max() < 1e-14
    assert np.abs(C).max() > 0.01 * h


@pytest.mark.parametrize("pde", ["diffusion", "advection_diffusion_reaction"])
def test_fem_operator_is_consistent(pde):
    """-Mm^{-1}(mu K + C) - r applied to cos(pi x) cos(pi y) approaches
    mu Lap f - u . grad f - r f at second order on the uniform mesh."""
    mu, r, adv = inputs.PAPER_PDES[pde]
    errs = []
    for n in (11, 23):
        w = inputs.paper_pde(pde, n=n, N=4, discretization="fem")
        h = 1.0 / (n + 1)
        xs = -0.5 + h * np.arange(1, n + 1)
        X, Y = np.meshgrid(xs, xs, indexing="xy")
        f = np.cos(np.pi * X) * np.cos(np.pi * Y)
        fx = -np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)
        fy = -np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y)
        Lf = -2 * np.pi ** 2 * mu * f - r * f
        if adv:
            Lf = Lf - ((-Y) * fx + X * fy)
        got = (w.A @ f.ravel()).reshape(n, n)
        # in the middle half of the square (the consistent mass matrix spreads
        # the first-order boundary error of the convection term a few rows in)
        q = n // 4
        errs.append(np.abs(got - Lf)[q:-q, q:-q].max() / np.abs(Lf).max())
    assert errs[1] < errs[0] / 3.0 and errs[1] < 5e-3


def test_stored_serial_slices_agree_with_the_stored_oracle_run():
    """The full-slice fixture and the sampled oracle run were written by the
    same oracle script: slice 0 is the workload's y0, and every 64th slice
    holds the sampled serial values of the JSON fixture."""
    import json
    import os
    gdir = os.path.join(os.path.dirname(__file__), "golden")
    lam = np.load(os.path.join(gdir, "oracle_serial_heat2d_128_N512_every32.npy"))
    g = json.load(open(os.path.join(gdir, "oracle_solve_heat2d_128_N512.json")))
    assert lam.shape == (17, 128 * 128)
    np.testing.assert_array_equal(lam[0], inputs.heat2d().y0[0])
    got = np.array([[lam[n // 32, i] for i in g["sample_points"]] for n in g["sample_slices"]])
    np.testing.assert_allclose(got, np.array(g["serial_samples"]), rtol=1e-14, atol=1e-300)
