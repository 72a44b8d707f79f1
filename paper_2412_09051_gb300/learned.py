"""Learned collision correction: data generation, training and evaluation
driver (argument marshalling and data plumbing only; every step of the method,
the features, the training and the corrected step run in libsllbm.so).

Pairs come from plain fine runs (order-2 cells, D2Q19, FP32) coarse-grained
2x by injection (coarse node k is fine node 2k in each direction): the coarse
state at t is the injected fine state, its plain coarse step (time step 2 dt)
gives f_plain and the features z, and the target is the injected fine state
two fine steps later.  R = (f_fine(t + 2 dt) - f_plain) / w.
"""
import ctypes as C
import time

import numpy as np

from . import capi
from .sim import Sim, _ptr

H = 64


def n_params(Q):
    return 128 * Q + 4224 + Q


def init_params(Q, seed):
    """Seeded Glorot-uniform initial weights, zero biases (flattened W1|b1|W2|b2|W3|b3)."""
    r = np.random.Generator(np.random.Philox(int(seed)))

    def glorot(o, i):
        a = np.sqrt(6.0 / (o + i))
        return r.uniform(-a, a, size=(o, i))
    parts = [glorot(H, Q), np.zeros(H), glorot(H, H), np.zeros(H), 0.1 * glorot(Q, H), np.zeros(Q)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def inject(f, n_fine):
    """Coarse-grain [Q, n_fine^2] populations by injection onto [Q, (n_fine/2)^2]."""
    Q = f.shape[0]
    return np.ascontiguousarray(f.reshape(Q, n_fine, n_fine)[:, ::2, ::2].reshape(Q, -1))


def case_cfg(base, cells, kind, mach, seed):
    from workloads.configs import get_config
    cfg = get_config("learned", cells=cells)
    cfg["init"] = dict(kind=kind, mach=mach, seed=seed)
    return cfg


class Trainer:
    def __init__(self, sim, params):
        L = capi.lib()
        h = C.c_void_p()
        p = np.ascontiguousarray(params, dtype=np.float32)
        capi.check(L.sllbm_train_create(sim.h, p.ctypes.data_as(C.c_void_p), C.byref(h)))
        self.h = h
        self.Q = sim.Q

    def _chk(self, rc):
        if rc != 0:
            msg = capi.lib().sllbm_train_last_error(self.h)
            raise capi.SllbmError(rc, msg.decode() if msg else "")

    def set_data(self, Z, R, max_degree=0):
        Z = np.ascontiguousarray(Z, dtype=np.float32)
        R = np.ascontiguousarray(R, dtype=np.float32)
        self._chk(capi.lib().sllbm_train_set_data(self.h, _ptr(Z)[0], _ptr(R)[0], C.c_int64(len(Z)),
                                                  int(max_degree), 0))

    def scales(self):
        s = np.zeros(self.Q, np.float32)
        sig = C.c_float()
        self._chk(capi.lib().sllbm_train_scales(self.h, _ptr(s)[0], C.byref(sig)))
        return s, sig.value

    def epoch(self, batch, lr):
        loss = C.c_float()
        self._chk(capi.lib().sllbm_train_epoch(self.h, batch, C.c_float(lr), C.byref(loss)))
        return loss.value

    def path(self, path):
        """capi.MLP_TENSOR (default) or capi.MLP_SIMT: where the forward and
        backward passes run."""
        self._chk(capi.lib().sllbm_train_path(self.h, path))

    def grads(self, offset, count):
        g = np.zeros(n_params(self.Q), np.float32)
        loss = C.c_float()
        self._chk(capi.lib().sllbm_train_grads(self.h, C.c_int64(offset), count, _ptr(g)[0], C.byref(loss)))
        return g, loss.value

    def params(self):
        p = np.zeros(n_params(self.Q), np.float32)
        self._chk(capi.lib().sllbm_train_params(self.h, _ptr(p)[0]))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._chk(capi.lib().sllbm_train_set_params(self.h, _ptr(p)[0]))

    def export(self):
        Q = self.Q
        w = np.zeros(2 * H * Q + H * H, np.uint16)
        b = np.zeros(2 * H + Q, np.float32)
        self._chk(capi.lib().sllbm_train_export(self.h, _ptr(w)[0], _ptr(b)[0]))
        return w, b

    def close(self):
        if getattr(self, "h", None):
            capi.lib().sllbm_train_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_mlp(sim, w_bf16, biases, s_in, sigma, enable=True):
    w_bf16 = np.ascontiguousarray(w_bf16, dtype=np.uint16)
    biases = np.ascontiguousarray(biases, dtype=np.float32)
    s_in = np.ascontiguousarray(s_in, dtype=np.float32)
    sim._call("sllbm_mlp_set", _ptr(w_bf16)[0], _ptr(biases)[0], _ptr(s_in)[0], C.c_float(sigma),
              1 if enable else 0)


def install_params(sim, params, s_in, sigma):
    """Installs flattened FP32 parameters (W1|b1|W2|b2|W3|b3) as the correction:
    the library's trainer rounds the weights to BF16."""
    tr = Trainer(sim, params)
    w, b = tr.export()
    tr.close()
    set_mlp(sim, w, b, s_in, sigma)


def step_features(sim):
    z = np.zeros((sim.N, sim.Q), np.float32)
    sim._call("sllbm_step_features", _ptr(z)[0], 0)
    return z


def generate_pairs(cases, fine_cells=128, snapshots=8, stride=4, spinup=4):
    """(Z [M, Q], R [M, Q]) from plain fine runs of the given (kind, mach, seed) cases."""
    from workloads import initial_fields
    Zs, Rs = [], []
    for kind, mach, seed in cases:
        cf = case_cfg(None, fine_cells, kind, mach, seed)
        cc = case_cfg(None, fine_cells // 2, kind, mach, seed)
        fine = Sim(cf, precision="fp32")
        coarse = Sim(cc, precision="fp32")
        _, w, _ = coarse.velocity_set()
        nf = fine.info.nodes[0]
        rho, u, T = initial_fields(cf, fine.node_coords())
        fine.init_state(rho, u, T)
        fine.step(spinup)
        for _ in range(snapshots):
            f, g = fine.get_state()
            coarse.set_state(inject(f, nf), inject(g, nf))
            z = step_features(coarse)
            fp, _ = coarse.get_state()
            fine.step(2)
            f2, _ = fine.get_state()
            R = (inject(f2, nf) - fp) / w[:, None]
            Zs.append(z)
            Rs.append(R.T.astype(np.float32))
            fine.step(max(stride - 2, 0))
        fine.close()
        coarse.close()
    return np.concatenate(Zs), np.concatenate(Rs)


def train(sim, Z, R, epochs=60, batch=512, lr=2e-3, seed=0, max_degree=3, apply_scale=0.5):
    """Train on (Z, R); the target keeps its stress and heat-flux moments
    (degree <= max_degree) so the network does not fit high-order noise.
    The installed correction is apply_scale times the one-step prediction:
    a full-strength correction overshoots in multi-step rollouts (chosen on
    validation vortex / shear-layer cases that the tests do not evaluate)."""
    r = np.random.Generator(np.random.Philox(seed))
    perm = r.permutation(len(Z))
    tr = Trainer(sim, init_params(sim.Q, seed))
    tr.set_data(Z[perm], R[perm], max_degree)
    losses = []
    for e in range(epochs):
        lr_e = lr * (0.5 * (1 + np.cos(np.pi * e / epochs)))
        losses.append(tr.epoch(batch, max(lr_e, lr * 0.02)))
    w, b = tr.export()
    s_in, sigma = tr.scales()
    tr.close()
    return dict(w=w, b=b, s_in=s_in, sigma=sigma * apply_scale, losses=losses)


def evaluate(model, case, fine_cells=128, steps=20, spinup=4):
    """Errors of the plain and the learned coarse run against the injected fine
    FP64 reference after `steps` coarse steps, and GPU time per coarse step."""
    import torch
    from workloads import initial_fields
    kind, mach, seed = case
    cf = case_cfg(None, fine_cells, kind, mach, seed)
    cc = case_cfg(None, fine_cells // 2, kind, mach, seed)
    ref = Sim(cf, precision="fp64")
    nf = ref.info.nodes[0]
    rho, u, T = initial_fields(cf, ref.node_coords())
    ref.init_state(rho, u, T)
    ref.step(spinup)
    f0, g0 = ref.get_state()
    ref.step(2 * steps)
    fr, gr = ref.get_state()
    rr, ur, Tr = ref.moments()
    sel = np.arange(ref.N).reshape(nf, nf)[::2, ::2].ravel()
    ref_moments = (rr[sel], ur[sel], Tr[sel])
    out = {}
    for name, learned in (("plain", False), ("learned", True)):
        s = Sim(cc, precision="fp32")
        if learned:
            set_mlp(s, model["w"], model["b"], model["s_in"], model["sigma"])
        s.set_state(inject(f0, nf), inject(g0, nf))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(steps)
        s.sync()
        dt = (time.perf_counter() - t0) / steps
        f, g = s.get_state()
        _, w, _ = s.velocity_set()
        fi = inject(fr, nf)
        rho_s, u_s, T_s = s.moments()
        rho_r, u_r, T_r = ref_moments
        out[name] = dict(err_rho=float(np.sqrt(np.mean((rho_s - rho_r) ** 2))),
                         err_u=float(np.sqrt(np.mean((u_s - u_r) ** 2))),
                         err_T=float(np.sqrt(np.mean((T_s - T_r) ** 2))),
                         err_f=float(np.sqrt(np.mean(((f - fi) / w[:, None]) ** 2))),
                         s_per_step=dt)
        s.close()
    ref.close()
    return out


def _resample(a, n_to):
    """Periodic Fourier resampling of node fields [..., n, n] (uniform nodes,
    x fastest) onto an n_to x n_to grid over the same box (evaluation only)."""
    n = a.shape[-1]
    F = np.fft.fft2(a, axes=(-2, -1))
    k = min(n, n_to) // 2
    G = np.zeros(a.shape[:-2] + (n_to, n_to), dtype=complex)
    for sy in (slice(0, k), slice(-k, None)):
        for sx in (slice(0, k), slice(-k, None)):
            G[..., sy, sx] = F[..., sy, sx]
    return np.fft.ifft2(G, axes=(-2, -1)).real * (n_to * n_to) / (n * n)


def evaluate_equal_cost(model, case, fine_cells=128, steps=10, spinup=4, mid_cells=80):
    """The learned coarse run against a plain run of about the same GPU cost:
    plain and learned at fine_cells/2 cells (`steps` steps), and plain at
    mid_cells cells whose step count reaches the same time (cost about
    (mid/coarse)^3 the plain coarse run in 2D).  Errors of rho, u, T against
    the FP64 fine reference at each run's own nodes (the reference resampled
    by Fourier interpolation, the box being periodic), and GPU seconds per run."""
    import torch
    from workloads import initial_fields
    kind, mach, seed = case
    cf = case_cfg(None, fine_cells, kind, mach, seed)
    cc = case_cfg(None, fine_cells // 2, kind, mach, seed)
    cm = case_cfg(None, mid_cells, kind, mach, seed)
    t_end = steps * cc["dt"]
    m_steps = int(round(t_end / cm["dt"]))
    cm["dt"] = t_end / m_steps
    ref = Sim(cf, precision="fp64")
    nf = ref.info.nodes[0]
    ref.init_state(*initial_fields(cf, ref.node_coords()))
    ref.step(spinup)
    f0, g0 = ref.get_state()
    ref.step(int(round(t_end / cf["dt"])))
    rr, ur, Tr = ref.moments()
    out = {}
    runs = (("plain_coarse", cc, False, steps), ("learned_coarse", cc, True, steps),
            ("plain_mid", cm, False, m_steps))
    for name, cfg, learned, n_steps in runs:
        s = Sim(cfg, precision="fp32")
        n = s.info.nodes[0]
        Q = f0.shape[0]
        if learned:
            set_mlp(s, model["w"], model["b"], model["s_in"], model["sigma"])
        fi = _resample(f0.reshape(Q, nf, nf), n).reshape(Q, -1)
        gi = _resample(g0.reshape(Q, nf, nf), n).reshape(Q, -1)
        s.set_state(fi, gi)
        s.step(1)                                    # warm-up launch outside the timing
        s.set_state(fi, gi)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(n_steps)
        s.sync()
        dt = time.perf_counter() - t0
        rho_s, u_s, T_s = s.moments()
        rho_r = _resample(rr.reshape(nf, nf), n).ravel()
        T_r = _resample(Tr.reshape(nf, nf), n).ravel()
        u_r = np.stack([_resample(ur[:, d].reshape(nf, nf), n).ravel() for d in range(2)], axis=1)
        out[name] = dict(cells=cfg["mesh"]["cells"][0], steps=n_steps,
                         err_rho=float(np.sqrt(np.mean((rho_s - rho_r) ** 2))),
                         err_u=float(np.sqrt(np.mean((u_s - u_r) ** 2))),
                         err_T=float(np.sqrt(np.mean((T_s - T_r) ** 2))),
                         gpu_s=dt)
        s.close()
    ref.close()
    return out


def frontier(model, case, coarse_cells=64, plain_factors=(1.0, 1.25, 1.5), steps=10, spinup=4, repeats=3):
    """Cost-error frontier of the plain method against the learned point:
    plain runs at coarse_cells times each factor (time step scaled with the
    cell size, step counts reaching the same time) and the learned run at
    coarse_cells, each started from the FP64 reference at twice the coarse
    resolution after `spinup` steps (Fourier resampled) and compared with it
    at the end (rho, u, T errors at each run's own nodes); GPU time of each
    run, the best of `repeats` timed repetitions after a warm-up launch."""
    import torch
    from workloads import initial_fields
    kind, mach, seed = case
    fine_cells = 2 * coarse_cells
    cf = case_cfg(None, fine_cells, kind, mach, seed)
    cc = case_cfg(None, coarse_cells, kind, mach, seed)
    t_end = steps * cc["dt"]
    ref = Sim(cf, precision="fp64")
    nf = ref.info.nodes[0]
    ref.init_state(*initial_fields(cf, ref.node_coords()))
    ref.step(spinup)
    f0, g0 = ref.get_state()
    ref.step(int(round(t_end / cf["dt"])))
    rr, ur, Tr = ref.moments()
    ref.close()
    runs = [(f"plain_x{fac:g}", int(round(coarse_cells * fac)), False) for fac in plain_factors]
    runs.append(("learned_x1", coarse_cells, True))
    out = {}
    for name, cells, learned in runs:
        cfg = case_cfg(None, cells, kind, mach, seed)
        n_steps = int(round(t_end / cfg["dt"]))
        cfg["dt"] = t_end / n_steps
        s = Sim(cfg, precision="fp32")
        n = s.info.nodes[0]
        Q = f0.shape[0]
        if learned:
            set_mlp(s, model["w"], model["b"], model["s_in"], model["sigma"])
        fi = _resample(f0.reshape(Q, nf, nf), n).reshape(Q, -1)
        gi = _resample(g0.reshape(Q, nf, nf), n).reshape(Q, -1)
        best = None
        for _ in range(repeats):
            s.set_state(fi, gi)
            s.step(1)                                # warm-up launch outside the timing
            s.set_state(fi, gi)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.step(n_steps)
            s.sync()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        rho_s, u_s, T_s = s.moments()
        rho_r = _resample(rr.reshape(nf, nf), n).ravel()
        T_r = _resample(Tr.reshape(nf, nf), n).ravel()
        u_r = np.stack([_resample(ur[:, d].reshape(nf, nf), n).ravel() for d in range(2)], axis=1)
        out[name] = dict(cells=cells, steps=n_steps, nodes=int(s.N), kernel=s.step_kernel(),
                         err_rho=float(np.sqrt(np.mean((rho_s - rho_r) ** 2))),
                         err_u=float(np.sqrt(np.mean((u_s - u_r) ** 2))),
                         err_T=float(np.sqrt(np.mean((T_s - T_r) ** 2))),
                         gpu_s=best)
        s.close()
    return out
