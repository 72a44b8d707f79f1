"""Workload configurations (plain numbers).

Units: gas constant R = 1, lattice reference state rho0 = T0 = 1, c_v = 1/(gamma-1),
speed of sound c = sqrt(gamma T).  Mesh `kind`: 0 box, 1 channel, 2 mixing
layer, 3 NACA O-grid.  Boundary `kind`: 0 periodic, 1 equilibrium,
2 bounce-back, 3 isothermal wall, 4 outlet, 5 far field (equilibrium upstream
of mid-chord, outlet downstream).  Boundary 0 is the low-y side (wall of the
O-grid), boundary 1 the high-y side (far field of the O-grid).
"""
import math

SQRT_GAMMA = math.sqrt(1.4)


def _bc(kind, rho=1.0, u=(0.0, 0.0, 0.0), T=1.0):
    return dict(kind=kind, rho=rho, u=tuple(u), T=T)


def _taylor_green(cells=32, p=2, steps=100, precision="fp64"):
    U = 0.3 * SQRT_GAMMA                      # Ma = 0.3 at T0 = 1
    L = 2.0 * math.pi
    return dict(
        name=f"tgv2d_{cells}x{cells}_p{p}", velset="D2Q19",
        mesh=dict(kind=0, p=p, cells=(cells, cells), length=(L, L), stretch=1.0, central=0),
        dt=0.02, gamma=1.4, Pr=1.0, mu_ref=U * 1.0 / 100.0, T_ref=1.0, mu_exp=0.0,
        bcs=[_bc(0), _bc(0)], precision=precision, steps=steps,
        init=dict(kind="taylor_green", U=U))


def _naca(cells=(256, 128), p=3, precision="fp32"):
    U = 1.5 * SQRT_GAMMA                      # Ma = 1.5 free stream at T = 1
    return dict(
        name=f"naca0012_ogrid_{cells[0]}x{cells[1]}_p{p}", velset="D2Q19",
        mesh=dict(kind=3, p=p, cells=tuple(cells), length=(1.0, 20.0), stretch=1.05, central=0,
                  thickness=0.12),
        dt=1.5e-4, gamma=1.4, Pr=1.0, mu_ref=U * 1.0 / 1.0e4, T_ref=1.0, mu_exp=0.0,
        bcs=[_bc(2), _bc(5, 1.0, (U, 0.0, 0.0), 1.0)], precision=precision, steps=1000,
        init=dict(kind="naca_freestream", U=U))


def _channel(cells=(64, 48, 48), p=2, precision="fp32", Tw=0.5):
    # Ma_b = 1.5 with respect to the wall sound speed sqrt(gamma T_w).  The wall
    # temperature sits below the lattice reference temperature T0 = 1 so that
    # the centre-line speed stays within the range the order-4 equilibrium of
    # the 45-velocity set handles stably (|u| / sqrt(T0) < 2).
    ub = 1.5 * math.sqrt(1.4 * Tw)
    h = 1.0
    return dict(
        name=f"channel3d_{cells[0]}x{cells[1]}x{cells[2]}_p{p}", velset="D3Q45",
        mesh=dict(kind=1, p=p, cells=tuple(cells),
                  length=(4.0 * math.pi * h, 2.0 * h, 4.0 / 3.0 * math.pi * h), stretch=2.0, central=0),
        dt=8.0e-4, gamma=1.4, Pr=0.7, mu_ref=1.0 * ub * h / 3000.0, T_ref=Tw, mu_exp=0.7,
        bcs=[_bc(3, 1.0, (0, 0, 0), Tw), _bc(3, 1.0, (0, 0, 0), Tw)], precision=precision,
        steps=1000, init=dict(kind="channel_laminar", ub=ub, amp=0.10, seed=1234, T=Tw))


def _mixing(cells=(96, 64, 48), p=2, mac=0.7, precision="fp32"):
    du = 2.0 * mac * SQRT_GAMMA              # Ma_c = du / (2 c) with T0 = 1 on both streams
    return dict(
        name=f"mixing3d_{cells[0]}x{cells[1]}x{cells[2]}_p{p}_mac{mac}", velset="D3Q45",
        mesh=dict(kind=2, p=p, cells=tuple(cells), length=(345.0, 172.0, 86.0), stretch=1.1,
                  central=cells[1] // 2),
        dt=0.02, gamma=1.4, Pr=0.71, mu_ref=du * 1.0 / 640.0, T_ref=1.0, mu_exp=0.0,
        bcs=[_bc(1, 1.0, (-0.5 * du, 0, 0), 1.0), _bc(1, 1.0, (0.5 * du, 0, 0), 1.0)],
        precision=precision, steps=1000, init=dict(kind="mixing_layer", du=du, amp=0.05, seed=1234))


def _learned(cells=128, p=2, precision="fp32"):
    cells = int(cells[0]) if isinstance(cells, (tuple, list)) else int(cells)   # square box
    L = 2.0 * math.pi
    return dict(
        name=f"learned2d_{cells}x{cells}_p{p}", velset="D2Q19",
        mesh=dict(kind=0, p=p, cells=(cells, cells), length=(L, L), stretch=1.0, central=0),
        dt=0.012 * 64 / cells, gamma=1.4, Pr=1.0, mu_ref=2.0e-3, T_ref=1.0, mu_exp=0.0,
        bcs=[_bc(0), _bc(0)], precision=precision, steps=200,
        init=dict(kind="isentropic_vortex", mach=0.6, seed=0))


CONFIGS = {
    "tgv2d": _taylor_green(),
    "naca": _naca(),
    "channel": _channel(),
    "mixing": _mixing(),
    "learned": _learned(),
}


def get_config(name, **over):
    """Return a config by name; keyword overrides rebuild it with other sizes."""
    builders = dict(tgv2d=_taylor_green, naca=_naca, channel=_channel, mixing=_mixing,
                    learned=_learned)
    if over:
        return builders[name](**over)
    return dict(CONFIGS[name])
