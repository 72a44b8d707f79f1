"""Helpers that build oracle cases from workload configs (test infrastructure)."""
import numpy as np

from oracle import step as st
from oracle.departure import trace
from oracle.mesh import Mesh
from oracle.velocity_sets import custom_set, velocity_set


def oracle_case(cfg):
    m = cfg["mesh"]
    mesh = Mesh(m["kind"], m["p"], m["cells"], m["length"], m.get("stretch", 1.0), m.get("central", 0),
                m.get("thickness", 0.12), vertices=m.get("vertices"),
                periodic_y=all(b["kind"] == 0 for b in cfg["bcs"]))
    if cfg["velset"] == "CUSTOM":
        xi, w, opp = custom_set(cfg["velset_xi"], cfg["velset_w"])
    else:
        xi, w, opp = velocity_set(cfg["velset"])
    par = st.Params(cfg["dt"], cfg["gamma"], cfg["Pr"], cfg["mu_ref"], cfg["T_ref"], cfg["mu_exp"], cfg["bcs"])
    rec = trace(mesh, xi, opp, cfg["dt"], cfg["bcs"])
    return mesh, xi, w, opp, par, rec


def box_cfg(cells=(8, 8), p=2, L=(1.0, 1.0), dt=0.01, velset="D2Q19", mu=0.01, Pr=1.0, mu_exp=0.0):
    D = len(cells)
    bc = dict(kind=0, rho=1.0, u=(0.0, 0.0, 0.0), T=1.0)
    return dict(name="box", velset=velset, mesh=dict(kind=0, p=p, cells=tuple(cells), length=tuple(L)),
                dt=dt, gamma=1.4, Pr=Pr, mu_ref=mu, T_ref=1.0, mu_exp=mu_exp, bcs=[bc, bc],
                precision="fp64", init=dict(kind="taylor_green", U=0.1))


def random_neq_state(xi, w, cv, N, seed, amp=0.02):
    """Equilibrium of random (rho, u, T) plus a seeded non-equilibrium perturbation
    (zero-mean is not enforced: collision must conserve whatever moments it has)."""
    from oracle.equilibrium import feq, geq
    from workloads.fields import random_state_perturbation
    rng = np.random.default_rng(seed)
    D = xi.shape[1]
    rho = rng.uniform(0.8, 1.2, N)
    u = rng.uniform(-0.5, 0.5, (N, D))
    T = rng.uniform(0.8, 1.2, N)
    f = feq(rho, u, T, xi, w) + random_state_perturbation(len(xi), N, seed + 1, amp) * w[:, None]
    g = geq(rho, u, T, xi, w, cv) + random_state_perturbation(len(xi), N, seed + 2, amp) * w[:, None]
    return f, g
