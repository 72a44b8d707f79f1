"""One SLLBM time step (Sec. 3.1 Eq. 1, Sec. 3.3), FP64 oracle.
TEST INFRASTRUCTURE ONLY.

State: post-collision nodal populations f, g [Q, N] (full values, FP64).
One step:
  1. stream    interpolate f_src, g_src at each departure record with the
               cell's Lagrange basis (Eq. intf and the streamed-value formula
               of Sec. 3.1); boundary records per Sec. 3.3
  2. moments   rho = sum f, rho u = sum zeta f, 2 rho E = sum |zeta|^2 f + g,
               with 2 rho E = rho |u|^2 + 2 rho c_v T (Sec. 3.1 moments)
  3. thermal   at nodes with an isothermal-wall trajectory:
               f += f^eq(rho,u,T_w) - f^eq(rho,u,T), g likewise (Eq. thermalBC)
  4. collide   h' = h - (1/tau)(h - h^eq) + (1/tau - 1/tau_Pr) h^*  (Eq. 1)
               tau = mu / (p dt) + 1/2 with p = rho T (R = 1),
               tau_Pr = (tau - 1/2)/Pr + 1/2                         (Sec. 3.1)
Readings (the paper is silent; see the design notes):
  * collision at the arrival point on the streamed values;
  * tau in time-step units: tau = mu/(p dt) + 1/2;
  * h^* (quasi-equilibrium part, Pr != 1) is zero for f and, for g,
    g*_i = w_i zeta_i . (2 q^neq) with the central non-equilibrium heat flux
    q^neq_a = 1/2 sum_i (zeta_i - u)_a [|zeta_i - u|^2 f^neq_i + g^neq_i],
    so that q relaxes with 1/tau_Pr and all other moments with 1/tau;
  * moving walls add 2 w_i rho_w zeta_i . u_w to the bounced f_i.
"""
import numpy as np

from .departure import REC_BB, REC_BB_ISO, REC_EQ
from .equilibrium import feq, geq


class Params:
    def __init__(self, dt, gamma=1.4, Pr=1.0, mu_ref=1e-3, T_ref=1.0, mu_exp=0.0, bcs=None, force=None):
        self.dt = float(dt)
        self.gamma = float(gamma)
        self.cv = 1.0 / (self.gamma - 1.0)
        self.Pr = float(Pr)
        self.mu_ref, self.T_ref, self.mu_exp = float(mu_ref), float(T_ref), float(mu_exp)
        self.bcs = bcs or [dict(kind=0, rho=1.0, u=(0.0, 0.0, 0.0), T=1.0)] * 2
        self.force = None if force is None else np.asarray(force, dtype=np.float64)


def init_equilibrium(rho, u, T, xi, w, cv):
    return feq(rho, u, T, xi, w), geq(rho, u, T, xi, w, cv)


def moments(f, g, xi, cv):
    rho = f.sum(0)
    j = xi.T @ f
    u = (j / rho).T
    e2 = ((xi ** 2).sum(1) @ f) + g.sum(0)
    T = (e2 - rho * (u ** 2).sum(1)) / (2.0 * rho * cv)
    return rho, u, T


def stream(mesh, rec, f, g, xi, w, par):
    """Streamed values for the arrival nodes the records were traced for."""
    Q, N = rec["kind"].shape
    D = mesh.D
    fs = np.zeros((Q, N))
    gs = np.zeros((Q, N))
    for i in range(Q):
        kind, src, cell = rec["kind"][i], rec["src"][i], rec["cell"][i]
        inter = kind != REC_EQ
        nn = np.nonzero(inter)[0]
        nodes = mesh.cell_nodes(cell[nn])
        L = mesh.basis(rec["xi"][i][nn])
        s = src[nn]
        fs[i, nn] = (L * f[s[:, None], nodes]).sum(1)
        gs[i, nn] = (L * g[s[:, None], nodes]).sum(1)
        # moving-wall momentum term on bounced populations
        bb = np.nonzero((kind == REC_BB) | (kind == REC_BB_ISO))[0]
        for b in (0, 1):
            sel = bb[rec["bid"][i][bb] == b]
            uw = np.array(par.bcs[b]["u"][:D], dtype=np.float64)
            fs[i, sel] += 2.0 * w[i] * par.bcs[b]["rho"] * float(xi[i] @ uw)
        eqn = np.nonzero(kind == REC_EQ)[0]
        for b in (0, 1):
            sel = eqn[rec["bid"][i][eqn] == b]
            if len(sel) == 0:
                continue
            bc = par.bcs[b]
            uw = np.array(bc["u"][:D], dtype=np.float64)[None, :]
            fe = feq(np.array([bc["rho"]]), uw, np.array([bc["T"]]), xi, w)[i, 0]
            fs[i, sel] = fe
            gs[i, sel] = bc["T"] * (2.0 * par.cv - D) * fe
    return fs, gs


def isothermal_nodes(rec, par):
    """Per node: wall temperature of the lowest velocity whose trajectory hit
    an isothermal wall, NaN where none did."""
    Q, N = rec["kind"].shape
    Tw = np.full(N, np.nan)
    for i in range(Q - 1, -1, -1):
        hit = rec["kind"][i] == REC_BB_ISO
        for n in np.nonzero(hit)[0]:
            Tw[n] = par.bcs[rec["bid"][i][n]]["T"]
    return Tw


def thermal_correction(fs, gs, xi, w, par, Tw):
    nn = np.nonzero(~np.isnan(Tw))[0]
    if len(nn) == 0:
        return fs, gs
    rho, u, T = moments(fs[:, nn], gs[:, nn], xi, par.cv)
    fs = fs.copy()
    gs = gs.copy()
    fs[:, nn] += feq(rho, u, Tw[nn], xi, w) - feq(rho, u, T, xi, w)
    gs[:, nn] += geq(rho, u, Tw[nn], xi, w, par.cv) - geq(rho, u, T, xi, w, par.cv)
    return fs, gs


def relaxation_times(rho, T, par):
    mu = par.mu_ref * (T / par.T_ref) ** par.mu_exp
    tau = mu / (rho * T * par.dt) + 0.5
    tau_pr = (tau - 0.5) / par.Pr + 0.5
    return tau, tau_pr


def heat_flux_neq(f, g, fe, ge, xi, u):
    c = xi[:, None, :] - u[None, :, :]             # [Q, N, D]
    c2 = (c ** 2).sum(2)
    return 0.5 * np.einsum("qnd,qn->nd", c, c2 * (f - fe) + (g - ge))


def collide(fs, gs, xi, w, par):
    rho, u, T = moments(fs, gs, xi, par.cv)
    fe = feq(rho, u, T, xi, w)
    ge = geq(rho, u, T, xi, w, par.cv)
    tau, tau_pr = relaxation_times(rho, T, par)
    om, om_pr = 1.0 / tau, 1.0 / tau_pr
    q = heat_flux_neq(fs, gs, fe, ge, xi, u)
    gstar = w[:, None] * (xi @ (2.0 * q).T)
    f1 = fs - om[None, :] * (fs - fe)
    g1 = gs - om[None, :] * (gs - ge) + (om - om_pr)[None, :] * gstar
    if par.force is not None and np.any(par.force != 0.0):
        # Kupershtokh exact-difference forcing after the collision (Sec. 4.3):
        # delta f_i = f_i^eq(rho, u + du, T) - f_i^eq(rho, u, T), du = F dt / rho
        du = par.force[None, : xi.shape[1]] * par.dt / rho[:, None]
        f1 = f1 + feq(rho, u + du, T, xi, w) - fe
    return f1, g1


def rescale_mass(f, g, target_mass):
    """Sec. 4.3: scale every population by target / current total mass (the
    nodal sum of rho); velocity and temperature are unchanged."""
    s = target_mass / f.sum()
    return f * s, g * s


def step(mesh, rec, f, g, xi, w, par, Tw=None, mlp=None):
    fs, gs = stream(mesh, rec, f, g, xi, w, par)
    if Tw is None:
        Tw = isothermal_nodes(rec, par)
    fs, gs = thermal_correction(fs, gs, xi, w, par, Tw)
    f1, g1 = collide(fs, gs, xi, w, par)
    if mlp is not None:
        f1 = f1 + mlp(fs, gs, f1, g1)
    return f1, g1


def step_sample_from_fields(mesh, rec, rho, u, T, xi, w, par):
    """One step for a subset of arrival nodes (records traced with `nodes=`),
    starting from the equilibrium of the full-mesh fields rho, u, T.  Only the
    support points that the records read are initialised."""
    Q = len(xi)
    need = rec["kind"] != REC_EQ
    cells = np.unique(rec["cell"][need])
    nodes = np.unique(mesh.cell_nodes(cells).ravel())
    f = np.zeros((Q, mesh.n_nodes))
    g = np.zeros((Q, mesh.n_nodes))
    f[:, nodes], g[:, nodes] = init_equilibrium(rho[nodes], u[nodes], T[nodes], xi, w, par.cv)
    Tw = isothermal_nodes(rec, par)
    fs, gs = stream(mesh, rec, f, g, xi, w, par)
    fs, gs = thermal_correction(fs, gs, xi, w, par, Tw)
    return collide(fs, gs, xi, w, par)
