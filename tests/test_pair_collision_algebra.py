"""The paired collision of the two-nodes-per-thread row-tile kernel, checked
on the CPU against the oracle (no GPU).

The kernel takes D3Q45 as 22 opposite pairs and the rest velocity (the
structure the library also checks on its own table before that kernel may
run) and computes the BGK collision with the quasi-equilibrium heat flux and
the exact-difference forcing in pair form: with c = xi_b . u for the base and
-c for the opposite, the equilibrium polynomial P1(+-c) = E(c^2) +- c O(c^2)
(Sec. 3.1, fourth-order Hermite equilibrium as a scalar polynomial in c),
momentum and heat-flux sums over xi_b times the pair's difference, the heat
flux as sum xi h - u sum h.  Here that algebra is restated in FP64 on
deviations from the rest state, as the kernel carries them, and compared
with the oracle's collide (Eq. 1 with its readings), so that a mistake in the
reformulation (a sign of the odd part, a dropped rest-velocity term, the
factor 2 of the heat flux) fails on the CPU.
"""
import numpy as np
import pytest

from oracle import step as ost
from oracle.velocity_sets import velocity_set

NPAIR = 22


# the pair layout of D3Q45 as the kernel indexes it
def base(k):
    return 1 + k if k < 6 else (7 + k if k < 16 else 17 + k)


def opp(b):
    return b + (10 if 13 <= b <= 22 else 6)


def zero(b):
    if b <= 12:
        return (b - 1) // 2
    if b <= 16:
        return -1
    return (b - 17) // 2 if b <= 32 else (b - 33) // 2


def slot(i):
    if i == 0:
        return 2 * NPAIR
    if i <= 6:
        return 2 * (i - 1)
    if i <= 12:
        return 2 * (i - 7) + 1
    if i <= 22:
        return 2 * (i - 7)
    if i <= 32:
        return 2 * (i - 17) + 1
    if i <= 38:
        return 2 * (i - 17)
    return 2 * (i - 23) + 1


def shell_of(s2):
    return {0.0: 0, 3.0: 1, 9.0: 2, 15.0: 3}[round(float(s2), 9)]


def test_d3q45_pair_structure():
    xi, w, op = velocity_set("D3Q45")
    Q = len(w)
    assert Q == 2 * NPAIR + 1
    assert np.all(xi[0] == 0.0)
    bases = [base(k) for k in range(NPAIR)]
    opps = [opp(b) for b in bases]
    assert sorted([0] + bases + opps) == list(range(Q))
    s2 = (xi ** 2).sum(1)
    for b, o in zip(bases, opps):
        assert op[b] == o and op[o] == b
        assert np.all(xi[o] == -xi[b])                       # exact negation
        z = zero(b)
        for d in range(3):
            if d == z:
                assert xi[b, d] == 0.0                       # exact zero, dropped by the kernel
            else:
                assert xi[b, d] != 0.0
        assert w[o] == w[b]
        assert shell_of(s2[b]) == shell_of(s2[o])
    # weights equal within a shell (the kernel takes one weight per shell)
    for sh in range(4):
        ws = {float(w[i]) for i in range(Q) if shell_of(s2[i]) == sh}
        assert len(ws) == 1
    # tensor-memory slots: a permutation, each pair in adjacent slots
    sl = [slot(i) for i in range(Q)]
    assert sorted(sl) == list(range(Q))
    for k, b in enumerate(bases):
        assert slot(b) == 2 * k and slot(opp(b)) == 2 * k + 1


def pair_collide(fs, gs, xi, w, par, force=None, mistake=None):
    """The kernel's paired collision, restated in FP64 on deviations from the
    rest state (f - w, g - w (2 c_v - D)); returns full populations.
    `mistake` plants one error in the restatement (tests of the check)."""
    Q, N = fs.shape
    D = 3
    cv = par.cv
    gf = 2.0 * cv - D
    df, dg = fs - w[:, None], gs - (w * gf)[:, None]
    bases = [base(k) for k in range(NPAIR)]
    s2 = (xi ** 2).sum(1)
    # moments over pairs
    rho_d = df[0].copy()
    j = np.zeros((D, N))
    e = dg[0].copy()
    for b in bases:
        o = opp(b)
        fsum, fdif = df[b] + df[o], df[b] - df[o]
        rho_d += fsum
        j += xi[b][:, None] * fdif[None, :]
        e += s2[b] * fsum + dg[b] + dg[o]
    rho = 1.0 + rho_d
    u = j / rho
    U = (u ** 2).sum(0)
    t = (e - rho * U - 2.0 * cv * rho_d) / (rho * 2.0 * cv)
    T = 1.0 + t
    mu = par.mu_ref * (T / par.T_ref) ** par.mu_exp
    tau = mu / (rho * T * par.dt) + 0.5
    om = 1.0 / tau
    om_pr = 1.0 / ((tau - 0.5) / par.Pr + 0.5)
    rhoT_d = rho_d + rho * t

    def coef(s, V):
        A, B, C, E = s - D, s - D - 2, s - D - 4, s * s - 2 * (D + 2) * s + D * (D + 2)
        k2 = 0.5 - 0.25 * V + 0.25 * t * C
        k1 = 1.0 - 0.5 * V + 0.5 * t * B
        k0 = -0.5 * V + 0.125 * V * V + 0.5 * t * A - 0.25 * t * V * B + 0.125 * t * t * E
        return k0, k1, k2

    if force is not None:
        v = u + (np.asarray(force)[:, None] * par.dt) / rho[None, :]
        V = (v ** 2).sum(0)
    out_f, out_g = np.empty_like(fs), np.empty_like(gs)
    q = np.zeros((D, N))
    hs = np.zeros(N)
    for b in bases:
        o = opp(b)
        k0, k1, k2 = coef(s2[b], U)
        c = xi[b] @ u
        c2 = c * c
        E = k0 + c2 * (k2 + c2 / 24.0)
        cO = c * (k1 + c2 / 6.0)
        Pb, Po = E + cO, (E + cO if mistake == "odd_sign" else E - cO)
        fnb = df[b] - w[b] * (rho * Pb + rho_d)
        fno = df[o] - w[b] * (rho * Po + rho_d)
        gnb = dg[b] - w[b] * gf * (rho * T * Pb + rhoT_d)
        gno = dg[o] - w[b] * gf * (rho * T * Po + rhoT_d)
        hb = (s2[b] + U - 2.0 * c) * fnb + gnb
        ho = (s2[b] + U + 2.0 * c) * fno + gno
        q += xi[b][:, None] * (hb - ho)[None, :]
        hs += hb + ho
        out_f[b], out_f[o] = df[b] - om * fnb, df[o] - om * fno
        out_g[b], out_g[o] = dg[b] - om * gnb, dg[o] - om * gno
        if force is not None:
            kf0, kf1, kf2 = coef(s2[b], V)
            cw = xi[b] @ v
            w2 = cw * cw
            dE = kf0 + w2 * (kf2 + w2 / 24.0) - E
            dO = cw * (kf1 + w2 / 6.0) - cO
            out_f[b] += w[b] * rho * (dE + dO)
            out_f[o] += w[b] * rho * (dE - dO)
    # the rest velocity: c = 0, P1 = k0
    k0, _, _ = coef(0.0, U)
    fn0 = df[0] - w[0] * (rho * k0 + rho_d)
    gn0 = dg[0] - w[0] * gf * (rho * T * k0 + rhoT_d)
    if mistake != "rest_heat":
        hs += U * fn0 + gn0
    out_f[0], out_g[0] = df[0] - om * fn0, dg[0] - om * gn0
    if force is not None:
        kf0, _, _ = coef(0.0, V)
        out_f[0] += w[0] * rho * (kf0 - k0)
    a = om - om_pr
    q = a[None, :] * (q - u * hs[None, :]) * (0.5 if mistake == "heat_half" else 1.0)
    for b in bases:
        wdq = w[b] * (xi[b] @ q)
        out_g[b] += wdq
        out_g[opp(b)] -= wdq
    return out_f + w[:, None], out_g + (w * gf)[:, None]


@pytest.mark.parametrize("forced", [False, True])
def test_pair_form_matches_oracle_collision(forced):
    xi, w, _ = velocity_set("D3Q45")
    rng = np.random.default_rng(2412)
    N = 300
    force = np.array([2e-3, -1e-3, 5e-4]) if forced else None
    par = ost.Params(0.05, gamma=1.4, Pr=0.71, mu_ref=2e-3, T_ref=0.9, mu_exp=0.7, force=force)
    rho = 1.0 + 0.05 * rng.standard_normal(N)
    u = 0.15 * rng.standard_normal((N, 3))
    T = 1.0 + 0.05 * rng.standard_normal(N)
    f, g = ost.init_equilibrium(rho, u, T, xi, w, par.cv)
    # off-equilibrium parts, so that the heat flux and the relaxation act
    f = f + 2e-3 * w[:, None] * rng.standard_normal(f.shape)
    g = g + 2e-3 * w[:, None] * rng.standard_normal(g.shape)
    f1, g1 = ost.collide(f, g, xi, w, par)
    p1, q1 = pair_collide(f, g, xi, w, par, force)
    scale = w[:, None]
    assert np.abs((p1 - f1) / scale).max() < 1e-11
    assert np.abs((q1 - g1) / scale).max() < 1e-11


@pytest.mark.parametrize("mistake", ["odd_sign", "rest_heat", "heat_half"])
def test_pair_form_check_catches_planted_mistakes(mistake):
    """The comparison is sharp: the odd part of the equilibrium with the base's
    sign for the opposite velocity, the rest velocity left out of the heat
    flux's u sum h term, or the heat flux halved (the oracle's q carries the
    factor 1/2 that the kernel's correction folds into 2 q) each fail it."""
    xi, w, _ = velocity_set("D3Q45")
    rng = np.random.default_rng(7)
    N = 50
    par = ost.Params(0.05, gamma=1.4, Pr=0.71, mu_ref=2e-3, T_ref=1.0, mu_exp=0.0)
    rho = 1.0 + 0.05 * rng.standard_normal(N)
    u = 0.15 * rng.standard_normal((N, 3))
    T = 1.0 + 0.05 * rng.standard_normal(N)
    f, g = ost.init_equilibrium(rho, u, T, xi, w, par.cv)
    f = f + 2e-3 * w[:, None] * rng.standard_normal(f.shape)
    g = g + 2e-3 * w[:, None] * rng.standard_normal(g.shape)
    f1, g1 = ost.collide(f, g, xi, w, par)
    p1, q1 = pair_collide(f, g, xi, w, par)
    assert max(np.abs((p1 - f1) / w[:, None]).max(), np.abs((q1 - g1) / w[:, None]).max()) < 1e-11
    p2, q2 = pair_collide(f, g, xi, w, par, mistake=mistake)
    err = max(np.abs((p2 - f1) / w[:, None]).max(), np.abs((q2 - g1) / w[:, None]).max())
    assert err > 1e-7, (mistake, err)


def heat_flux_from_moments(fs, gs, xi, w, par, shift=5.0):
    """The kernel's heat flux (unscaled: sum_i (xi_i - u)(|xi_i - u|^2 f^neq_i
    + g^neq_i)) from sums over the pairs of the deviations, taken before the
    isothermal correction: sum xi_b ((|xi|^2 - (D + 2) - g_f)(f_b - f_o) +
    g_b - g_o) + u ((D + 2 + g_f) rho_d - e + 2 rho U) - 2 M2 u, with M2 the
    second moments of the deviations and e their energy sum (`shift`: the
    D + 2 of the formula, changed only to test the check)."""
    D = 3
    gf = 2.0 * par.cv - D
    df, dg = fs - w[:, None], gs - (w * gf)[:, None]
    s2 = (xi ** 2).sum(1)
    N = fs.shape[1]
    rho_d, e = df[0].copy(), dg[0].copy()
    j, qx, M2 = np.zeros((D, N)), np.zeros((D, N)), np.zeros((D, D, N))
    for k in range(NPAIR):
        b = base(k)
        o = opp(b)
        fsum, fdif = df[b] + df[o], df[b] - df[o]
        rho_d += fsum
        j += xi[b][:, None] * fdif[None, :]
        e += s2[b] * fsum + dg[b] + dg[o]
        qx += xi[b][:, None] * ((s2[b] - shift - gf) * fdif + dg[b] - dg[o])[None, :]
        M2 += np.outer(xi[b], xi[b])[:, :, None] * fsum[None, None, :]
    rho = 1.0 + rho_d
    u = j / rho
    U = (u ** 2).sum(0)
    sc = (shift + gf) * rho_d - e + 2.0 * rho * U
    return (qx + u * sc[None, :] - 2.0 * np.einsum("abn,bn->an", M2, u)).T


def test_heat_flux_from_moments_matches_oracle():
    """The equilibrium's central third moment vanishes on D3Q45, so the heat
    flux of the quasi-equilibrium term is the central moment of the node's own
    populations; taken before the isothermal-wall correction (equilibria at
    the same rho and u, Eq. thermalBC) it equals the oracle's heat flux after
    it."""
    xi, w, _ = velocity_set("D3Q45")
    rng = np.random.default_rng(45)
    N = 200
    par = ost.Params(0.05, gamma=1.4, Pr=0.71, mu_ref=2e-3, T_ref=0.9, mu_exp=0.7)
    rho = 1.0 + 0.05 * rng.standard_normal(N)
    u = 0.2 * rng.standard_normal((N, 3))
    T = 1.0 + 0.08 * rng.standard_normal(N)
    f, g = ost.init_equilibrium(rho, u, T, xi, w, par.cv)
    f = f + 2e-3 * w[:, None] * rng.standard_normal(f.shape)
    g = g + 2e-3 * w[:, None] * rng.standard_normal(g.shape)
    Tw = np.where(rng.random(N) < 0.5, 1.0 + 0.1 * rng.standard_normal(N), np.nan)
    fc, gc = ost.thermal_correction(f, g, xi, w, par, Tw)
    r, uu, TT = ost.moments(fc, gc, xi, par.cv)
    fe, ge = ost.feq(r, uu, TT, xi, w), ost.geq(r, uu, TT, xi, w, par.cv)
    q_oracle = 2.0 * ost.heat_flux_neq(fc, gc, fe, ge, xi, uu)
    q = heat_flux_from_moments(f, g, xi, w, par)
    assert np.abs(q_oracle).max() > 1e-3
    assert np.abs(q - q_oracle).max() < 1e-12
    # the third moments shifted by D instead of D + 2 fail it (the result
    # moves by 2 u; the reference g_f cancels and cannot be tested this way)
    bad = heat_flux_from_moments(f, g, xi, w, par, shift=3.0)
    assert np.abs(bad - q_oracle).max() > 1e-2
