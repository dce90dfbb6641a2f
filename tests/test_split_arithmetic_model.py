"""The split RK4 step's arithmetic on a float32 model (CPU), against RK4 in
extended precision.

The 2D heat true residual steps u <- R(Z) u, Z = dt L, with the state in
float-float: the first-order term Z u in float-float, the higher-order terms
Z^2 u/2 + Z^3 u/6 + Z^4 u/24 in FP32 from a = fl(Z u).  With z = 8 nu dt /
h^2 >= ||Z||, those FP32 terms have size at most q(z) = z^2/2 + z^3/6 +
z^4/24 times |u|, so their rounding costs at most about 4 * 2^-24 q(z) |u|
per step.  The second form ("fold") leaves the low word out of the
float-float stencil and applies Z to it among the FP32 terms,
q = Z (u_lo + a/2 + (Z/6)(a + (Z/4) a)); its rounding scales the same way.
Both forms must stay within m times the per-step bound of the exact RK4
trajectory on white noise (the worst case) and far below it on smooth data.

The model rounds every operation to float32 as the kernels do (a fused
multiply-add is formed in float64 and rounded once to float32; the product
of two float32 values is exact in float64), with TwoSum for the error-free
sums.  It checks the arithmetic scheme, not the kernels.
"""
import numpy as np
import pytest

F32 = np.float32
LD = np.longdouble


def _fma(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(F32)


def _two_sum(a, b):
    s = (a + b).astype(F32)
    bb = (s - a).astype(F32)
    e = ((a - (s - bb).astype(F32)).astype(F32) + (b - bb).astype(F32)).astype(F32)
    return s, e


def _nbrs(u):
    p = np.zeros((u.shape[0] + 2, u.shape[1] + 2), dtype=u.dtype)
    p[1:-1, 1:-1] = u
    return p[:-2, 1:-1], p[2:, 1:-1], p[1:-1, :-2], p[1:-1, 2:]


def _lap32(x):
    n, s, w, e = _nbrs(x)
    t = ((n + s).astype(F32) + (w + e).astype(F32)).astype(F32)
    return _fma(np.full_like(x, -4.0), x, t)


def _split_step(uh, ul, c, fold):
    ch = F32(c)
    cl = F32(LD(c) - LD(ch))
    nh, sh, wh, eh = _nbrs(uh)
    ah, al = _two_sum(nh, sh)
    bh, bl = _two_sum(wh, eh)
    sh_, sl_ = _two_sum(ah, bh)
    dh = _fma(np.full_like(uh, -4.0), uh, sh_)
    dl = (LD(sh_) - 4 * LD(uh) - LD(dh)).astype(F32)          # dh's rounding error (exact)
    lo = ((al + bl).astype(F32) + (sl_ + dl).astype(F32)).astype(F32)
    if not fold:
        nl, sl, wl, el = _nbrs(ul)
        lw = ((nl + sl).astype(F32) + (wl + el).astype(F32)).astype(F32)
        lo = _fma(np.full_like(ul, -4.0), ul, (lo + lw).astype(F32))
    p = (ch * dh).astype(F32)
    e = _fma(np.full_like(uh, ch), dh, -p)
    e = _fma(np.full_like(uh, ch), lo, e)
    e = _fma(np.full_like(uh, cl), dh, e)
    s_h, s_l = _two_sum(uh, p)
    s_l = (s_l + (ul + e).astype(F32)).astype(F32)
    a = p
    a3 = _fma(np.full_like(a, F32(c / 4)), _lap32(a), a)
    if fold:
        y = _fma(np.full_like(a, F32(c / 6)), _lap32(a3), _fma(np.full_like(a, F32(0.5)), a, ul))
        q = (ch * _lap32(y)).astype(F32)
    else:
        a2 = _fma(np.full_like(a, F32(c / 3)), _lap32(a3), a)
        q = (F32(c / 2) * _lap32(a2)).astype(F32)
    h, l = _two_sum(s_h, q)
    l = (l + s_l).astype(F32)
    hi = (h + l).astype(F32)
    return hi, (l - (hi - h).astype(F32)).astype(F32)


def _rk4_exact(u, c, m):
    def L(x):
        n, s, w, e = _nbrs(x)
        return n + s + w + e - 4 * x
    for _ in range(m):
        z1 = c * L(u)
        z2 = c * L(z1)
        z3 = c * L(z2)
        z4 = c * L(z3)
        u = u + z1 + z2 / 2 + z3 / 6 + z4 / 24
    return u


def _errors(u0, c, m):
    u0 = LD(u0)
    ref = _rk4_exact(u0, LD(c), m)
    scale = float(np.abs(ref).max())
    out = {}
    for fold in (False, True):
        h = u0.astype(F32)
        l = (u0 - LD(h)).astype(F32)
        for _ in range(m):
            h, l = _split_step(h, l, c, fold)
        out[fold] = float(np.abs(LD(h) + LD(l) - ref).max()) / scale
    return out


def _case(z=0.052, n=32, m=50):
    """A 32^2 grid, m RK4 steps with z = 8 nu dt / h^2 (the 128^2 workload
    has z = 0.052; the library takes the split step up to z = 1/8)."""
    return n, z / 8, m


def _bound(c, m):
    z = 8 * c
    q = z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    return m * 4 * 2.0 ** -24 * q


@pytest.mark.parametrize("z", [0.052, 0.11])
def test_split_step_model_white_noise_within_the_bound(z):
    n, c, m = _case(z)
    assert 8 * c <= 0.125
    u0 = np.random.default_rng(5).standard_normal((n, n))
    err = _errors(u0, c, m)
    for fold in (False, True):
        assert err[fold] < _bound(c, m), (fold, err, _bound(c, m))
    # the two forms are of the same accuracy
    assert err[True] < 2 * err[False] + 1e-15


def test_split_step_model_smooth_data_far_below_the_bound():
    n, c, m = _case()
    x = np.arange(1, n + 1) / (n + 1)
    X, Y = np.meshgrid(x, x)
    u0 = np.exp(-((X - 0.4) ** 2 + (Y - 0.6) ** 2) / (2 * 0.08 ** 2)) + 0.5 * np.sin(np.pi * X) * np.sin(2 * np.pi * Y)
    err = _errors(u0, c, m)
    for fold in (False, True):
        assert err[fold] < 0.1 * _bound(c, m), (fold, err)


@pytest.mark.parametrize("z", [0.005, 0.052])
def test_split_step_model_needs_its_float_float_term(z):
    """A planted mistake: the first-order term formed in FP32 (its rounding
    error dropped) is over ten times less accurate than the split step on
    the same input, and at small z over ten times the split step's bound,
    so the model resolves what the float-float term buys."""
    n, c, m = _case(z)
    u0 = np.random.default_rng(6).standard_normal((n, n))
    ref = _rk4_exact(LD(u0), LD(c), m)
    h = u0.astype(F32)
    l = (LD(u0) - LD(h)).astype(F32)
    for _ in range(m):
        d = _lap32(h)
        p = (F32(c) * d).astype(F32)
        a3 = _fma(np.full_like(p, F32(c / 4)), _lap32(p), p)
        a2 = _fma(np.full_like(p, F32(c / 3)), _lap32(a3), p)
        q = (F32(c / 2) * _lap32(a2)).astype(F32)
        s_h, s_l = _two_sum(h, p)
        hh, ll = _two_sum(s_h, q)
        ll = (ll + (s_l + l).astype(F32)).astype(F32)
        h = (hh + ll).astype(F32)
        l = (ll - (h - hh).astype(F32)).astype(F32)
    err = float(np.abs(LD(h) + LD(l) - ref).max()) / float(np.abs(ref).max())
    assert err > 10 * max(_errors(u0, c, m).values())
    if z < 0.01:
        assert err > 10 * _bound(c, m)
