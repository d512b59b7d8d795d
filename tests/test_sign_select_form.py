"""The sign select of Eq. 2 in the iteration loop, on CPU.

For 1/4 <= alpha <= 4 the kernel takes u_eff^2 = t (t + rho |t|) with
t = sigma (y - delta), sigma^2 = (kp^2 + kn^2)/2 and rho = (kp^2 - kn^2)/
(kp^2 + kn^2) = (1 - alpha^2)/(1 + alpha^2), kp = 1/(c s), kn = alpha/(c s):
one FMA with |t| as an operand instead of two scaled residuals and their min.
This emulates that FP32 arithmetic (the per-curve rho, the per-slot FMAs,
each rounded once to float32) for a window's float32 sigma, and checks it
against u_eff^2 = sigma^2 (1 + rho sgn(u)) u^2 evaluated exactly in float64
with the exact rho.  sigma's own rounding (the reciprocal square root of the
mean square times a per-curve constant) is one factor common to every slot
of the window, as if c were perturbed by a few parts in 10^7, and is not part
of this bound.
  * the identity itself (both branches, both sides of alpha = 1);
  * the relative error of u_eff^2 stays within 4 + 3 (a^2 - 1)/2 units of
    roundoff (2^-24), a = max(alpha, 1/alpha): 4 from the roundings of t and
    of t + rho |t|, and rho's own (at most 3) grown by (a^2 - 1)/2 on the
    small side, where t + rho |t| is a difference; at a = 4 that is 26.5,
    1.6e-6 relative;
  * beyond a = 4 the same bound is broken for some alpha (why the kernel keeps
    the min form there);
  * a gap slot (far below every sample) gets weight exactly 0, also when t
    overflows to -inf and t + rho |t| is NaN.
"""
import numpy as np
import pytest

F32 = np.float32
ULP = 2.0 ** -24


def r32(v):
    return np.asarray(v, np.float64).astype(np.float32)


def fma32(a, b, c):
    """float32 FMA: the product of two float32 values is exact in float64."""
    with np.errstate(over="ignore", invalid="ignore"):
        return r32(np.float64(a) * np.float64(b) + np.float64(c))


def rho32(alpha):
    """rho as the kernel rounds it: two FMAs and a quotient."""
    a = F32(alpha)
    num = fma32(-a, a, F32(1.0))
    den = fma32(a, a, F32(1.0))
    return r32(np.float64(num) / np.float64(den))


def sigma32(alpha, c, s):
    """A window's sigma = sqrt((1 + alpha^2)/2)/(c s), rounded to float32."""
    return r32(np.sqrt(0.5 * (1.0 + np.float64(alpha) ** 2)) / (np.float64(c) * np.float64(s)))


def kernel_q2(y, delta, alpha, sg):
    """u_eff^2 as t * v (the kernel forms 1 - t v inside one FMA, so the
    product is exact there); returns (q2 in float64, z as the kernel rounds it)."""
    rho = rho32(alpha)
    c0 = r32(-np.float64(F32(delta)) * np.float64(sg))
    t = fma32(y, sg, c0)
    v = fma32(rho, np.abs(t), t)
    with np.errstate(over="ignore", invalid="ignore"):
        q2 = np.float64(t) * np.float64(v)
        z = fma32(-t, v, F32(1.0))
    z = np.where(np.isnan(z), F32(0.0), np.clip(z, F32(0.0), F32(1.0)))
    return q2, z


def exact_q2(y, delta, alpha, sg):
    """Eq. 2 in float64 for the same sigma: sigma^2 (1 + rho) u^2 above the
    trend, sigma^2 (1 - rho) u^2 below it, rho exact."""
    a2 = np.float64(F32(alpha)) ** 2
    rho = (1.0 - a2) / (1.0 + a2)
    u = np.float64(y) - np.float64(F32(delta))
    k2 = np.where(u < 0, 1.0 - rho, 1.0 + rho) * np.float64(sg) ** 2
    return k2 * u * u


def bound(a):
    return 4.0 + 1.5 * (a * a - 1.0)


def worst_rel_ulp(alpha, n=20000, seed=0):
    rng = np.random.default_rng(seed)
    c, s = 5.0, 1.3e-3
    y = r32(rng.normal(0.0, 4 * c * s, n))          # residuals about the median
    y = y[y != 0]
    sg = sigma32(alpha, c, s)
    q2, _ = kernel_q2(y, 0.0, alpha, sg)
    ref = exact_q2(y, 0.0, alpha, sg)
    return np.max(np.abs(q2 - ref) / ref) / ULP


def test_identity_selects_the_branch_by_sign():
    c, s = 5.0, 2e-3
    y = r32(np.array([3e-3, -3e-3, 1e-2, -1e-2, 4e-2, -4e-2]))
    for alpha in (0.25, 0.5, 1.0, 2.0, 3.0, 4.0):
        q2, _ = kernel_q2(y, 0.0, alpha, sigma32(alpha, c, s))
        # Eq. 2 itself: u/(c s) above the trend, alpha u/(c s) below it.
        u = np.float64(y) / (c * s)
        ref = np.where(u < 0, alpha * u, u) ** 2
        np.testing.assert_allclose(q2, ref, rtol=2e-6)
        # The two sides differ by alpha^2, below the trend is the stretched one.
        np.testing.assert_allclose(q2[1::2] / q2[0::2], alpha ** 2, rtol=4e-6)


@pytest.mark.parametrize("alpha", [0.25, 0.3, 0.5, 0.77, 1.0, 1.5, 2.0, 3.0, 3.7, 4.0])
def test_error_bound_where_the_kernel_uses_it(alpha):
    assert worst_rel_ulp(alpha) <= bound(max(alpha, 1.0 / alpha))


def test_bound_fails_for_large_asymmetry():
    # Somewhere past alpha = 4 the error leaves what the kernel accepts at 4.
    rel = [worst_rel_ulp(a) for a in np.linspace(9.0, 40.0, 32)]
    assert max(rel) > bound(4.0)


def test_weights_match_eq3_on_delta_shifted_residuals():
    rng = np.random.default_rng(1)
    c, s = 5.0, 1e-3
    y = r32(rng.normal(0.0, 3 * c * s, 5000))
    for alpha in (0.25, 2.0, 4.0):
        sg = sigma32(alpha, c, s)
        for delta in (0.0, 7e-4, -2e-3):
            _, z = kernel_q2(y, delta, alpha, sg)
            zref = np.clip(1.0 - exact_q2(y, delta, alpha, sg), 0.0, 1.0)
            # 1 - u_eff^2 loses at most a few ulp of u_eff^2 plus the final rounding.
            assert np.max(np.abs(np.float64(z) - zref)) < 3e-6


def test_gap_slots_get_zero_weight():
    kgap = F32(-2.0 ** 100)
    for alpha in (0.25, 0.5, 1.0, 2.0, 4.0):
        for s in (1e-3, 1e-30, 3e-38):            # tiny scales make t overflow to -inf
            y = r32(np.array([kgap - F32(1.0), kgap]))
            with np.errstate(over="ignore"):
                sg = sigma32(alpha, 5.0, s)
            _, z = kernel_q2(y, 0.0, alpha, sg)
            assert np.all(z == 0.0)
            assert np.all((z * z) == 0.0)
