"""Python-side handle on one SLLBM context (argument marshalling only).

Arrays are numpy (host) or torch CUDA tensors (device); torch is used only to
own device memory and streams.  All arithmetic happens in libsllbm.so.
"""
import ctypes as C

import numpy as np

from . import capi


def _ptr(a):
    """(pointer, on_device) for a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data_as(C.c_void_p), 0
    if a is None:
        return None, 0
    assert a.is_contiguous()
    return C.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0


def mesh_desc(cfg):
    """The mesh descriptor of a config.  The explicit kind (4) takes
    m["vertices"], one array of cells[d] + 1 coordinates per dimension; the
    arrays the descriptor points to are kept on it (``d._keep``)."""
    import numpy as np
    m = cfg["mesh"]
    d = capi.MeshDesc()
    d.kind = m["kind"]
    d.dim = len(m["cells"])
    d.p = m["p"]
    for k, c in enumerate(m["cells"]):
        d.cells[k] = c
        d.length[k] = m["length"][k]
    if m["kind"] == capi.MESH["explicit"]:
        d._keep = [np.ascontiguousarray(v, dtype=np.float64) for v in m["vertices"]]
        for k, v in enumerate(d._keep):
            d.vertices[k] = v.ctypes.data
    d.stretch = m.get("stretch", 1.0)
    d.central = m.get("central", 0)
    d.thickness = m.get("thickness", 0.12)
    for b in range(2):
        bc = cfg["bcs"][b]
        d.bc[b].kind = bc["kind"]
        d.bc[b].rho = bc["rho"]
        for k in range(3):
            d.bc[b].u[k] = bc["u"][k] if k < len(bc["u"]) else 0.0
        d.bc[b].T = bc["T"]
    return d


def params(cfg, precision=None, stream_mode=0, device=0, stream=None):
    p = capi.Params()
    p.dt = cfg["dt"]
    p.gamma = cfg["gamma"]
    p.Pr = cfg["Pr"]
    p.mu_ref = cfg["mu_ref"]
    p.T_ref = cfg["T_ref"]
    p.mu_exp = cfg["mu_exp"]
    prec = precision or cfg.get("precision", "fp32")
    p.precision = capi.FP64 if prec == "fp64" else capi.FP32
    p.stream_mode = stream_mode
    p.device = device
    p.stream = stream
    return p


def velset_desc(cfg):
    """The velocity-set descriptor of a config: cfg["velset"] names a set
    (D2Q9 .. D3Q125), or is "CUSTOM" with the caller's abscissae
    cfg["velset_xi"] [Q][D] and weights cfg["velset_w"] [Q].  Returns the
    descriptor and the arrays it points to (kept alive by the caller)."""
    import numpy as np
    d = capi.VelsetDesc()
    d.kind = capi.VELSET[cfg["velset"]]
    keep = ()
    if cfg["velset"] == "CUSTOM":
        xi = np.ascontiguousarray(cfg["velset_xi"], dtype=np.float64)
        w = np.ascontiguousarray(cfg["velset_w"], dtype=np.float64)
        d.Q, d.D = xi.shape
        d.xi = xi.ctypes.data
        d.w = w.ctypes.data
        keep = (xi, w)
    return d, keep


class Sim:
    """One library context built from a workload config dict."""

    def __init__(self, cfg, precision=None, stream_mode=0, device=0, stream=None):
        L = capi.lib()
        self.cfg = cfg
        self._desc = mesh_desc(cfg)
        self._par = params(cfg, precision, stream_mode, device, stream)
        h = C.c_void_p()
        vd, keep = velset_desc(cfg)
        rc = L.sllbm_create_desc(C.byref(self._desc), C.byref(vd), C.byref(self._par), C.byref(h))
        del keep
        if rc != capi.OK:
            msg = L.sllbm_last_error(None)
            raise capi.SllbmError(rc, msg.decode() if msg else "")
        self.h = h
        info = capi.Info()
        capi.check(L.sllbm_info(h, C.byref(info)), h)
        self.info = info
        self.N = info.n_nodes
        self.Q = info.Q
        self.D = info.dim
        self.fp64 = info.precision == capi.FP64

    def close(self):
        if getattr(self, "h", None):
            capi.lib().sllbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        return capi.check(getattr(capi.lib(), name)(self.h, *args), self.h)

    # ---------------------------------------------------------------- queries
    def node_coords(self):
        x = np.zeros((self.N, self.D))
        self._call("sllbm_node_coords", *_ptr(x))
        return x

    def velocity_set(self):
        xi = np.zeros((self.Q, self.D))
        w = np.zeros(self.Q)
        opp = np.zeros(self.Q, dtype=np.int32)
        self._call("sllbm_velocity_set", _ptr(xi)[0], _ptr(w)[0], _ptr(opp)[0])
        return xi, w, opp

    def stream(self):
        return capi.lib().sllbm_stream(self.h)

    # ---------------------------------------------------------------- state
    def init_state(self, rho, u, T):
        rho = np.ascontiguousarray(rho, dtype=np.float64) if isinstance(rho, np.ndarray) else rho
        u = np.ascontiguousarray(u, dtype=np.float64) if isinstance(u, np.ndarray) else u
        T = np.ascontiguousarray(T, dtype=np.float64) if isinstance(T, np.ndarray) else T
        pr, dev = _ptr(rho)
        self._call("sllbm_init_state", pr, _ptr(u)[0], _ptr(T)[0], dev)

    def get_state(self):
        f = np.zeros((self.Q, self.N))
        g = np.zeros((self.Q, self.N))
        self._call("sllbm_get_state", _ptr(f)[0], _ptr(g)[0], 0)
        return f, g

    def set_state(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        self._call("sllbm_set_state", _ptr(f)[0], _ptr(g)[0], 0)

    def get_state_raw(self, fg=None):
        """Native storage: deviations, interleaved (f, g) per population and node, [Q, N, 2]."""
        dt = np.float64 if self.fp64 else np.float32
        if fg is None:
            fg = np.zeros((self.Q, self.N, 2), dtype=dt)
        p, dev = _ptr(fg)
        self._call("sllbm_get_state_raw", p, dev)
        return fg

    def set_state_raw(self, fg):
        p, dev = _ptr(fg)
        self._call("sllbm_set_state_raw", p, dev)

    def get_x_layers(self, x0, nx, out=None):
        """Node layers x0 .. x0 + nx - 1, raw format [Q, rows, nx, 2] (numpy, or a
        torch CUDA tensor for a device copy)."""
        if out is None:
            rows = self.info.nodes[1] * (self.info.nodes[2] if self.D == 3 else 1)
            out = np.zeros((self.Q, rows, nx, 2), dtype=np.float64 if self.fp64 else np.float32)
        p, dev = _ptr(out)
        self._call("sllbm_get_x_layers", int(x0), int(nx), p, dev)
        return out

    def set_x_layers(self, x0, nx, buf):
        p, dev = _ptr(buf)
        self._call("sllbm_set_x_layers", int(x0), int(nx), p, dev)

    def step(self, n=1):
        self._call("sllbm_step", C.c_int64(n))

    def set_force(self, F):
        F = np.zeros(3) if F is None else np.ascontiguousarray(list(F) + [0.0] * (3 - len(F)), dtype=np.float64)
        self._call("sllbm_set_force", _ptr(F)[0])

    def rescale_mass(self, target):
        self._call("sllbm_rescale_mass", C.c_double(target))

    def step_controlled(self, n, target_momentum, force0, kp, ki, control_every=10, rescale_every=10,
                        target_mass=None):
        c = capi.Control(target_momentum, force0, kp, ki, control_every, rescale_every,
                         target_mass if target_mass is not None else float(self.N))
        F = np.zeros(3)
        self._call("sllbm_step_controlled", C.c_int64(n), C.byref(c), _ptr(F)[0])
        return F

    def sync(self):
        self._call("sllbm_sync")

    def step_kernel(self):
        """Name of the kernel the last step launched (sllbm_info)."""
        info = capi.Info()
        self._call("sllbm_info", C.byref(info))
        return info.step_kernel.decode()

    # ---------------------------------------------------------------- statistics
    def plane_profiles(self):
        """Reynolds / Favre plane averages (sllbm_plane_profiles): dict of
        y, rho, u, u_favre, T, p [N1(, D)] and R [N1, D, D]."""
        N1, D = self.info.nodes[1], self.D
        out = dict(y=np.zeros(N1), rho=np.zeros(N1), u=np.zeros((N1, D)), u_favre=np.zeros((N1, D)),
                   T=np.zeros(N1), p=np.zeros(N1), R=np.zeros((N1, D, D)))
        self._call("sllbm_plane_profiles", *[_ptr(out[k])[0] for k in ("y", "rho", "u", "u_favre", "T", "p", "R")])
        return out

    def stats_accumulate(self):
        """Adds the current state's plane means to the running sums (device, async)."""
        self._call("sllbm_stats_accumulate")

    def stats_reset(self):
        self._call("sllbm_stats_reset")

    def plane_profiles_mean(self):
        """Profiles of sllbm_plane_profiles from the time-averaged plane means;
        also returns the number of accumulated states under 'samples'."""
        N1, D = self.info.nodes[1], self.D
        out = dict(y=np.zeros(N1), rho=np.zeros(N1), u=np.zeros((N1, D)), u_favre=np.zeros((N1, D)),
                   T=np.zeros(N1), p=np.zeros(N1), R=np.zeros((N1, D, D)))
        n = C.c_int64()
        self._call("sllbm_plane_profiles_mean", *[_ptr(out[k])[0] for k in ("y", "rho", "u", "u_favre", "T", "p", "R")],
                   C.byref(n))
        out["samples"] = n.value
        return out

    def mixing_thickness(self, du, rho0=1.0):
        """(delta_theta, delta_omega) of the current state (sllbm_mixing_thickness)."""
        th, om = C.c_double(), C.c_double()
        self._call("sllbm_mixing_thickness", C.c_double(du), C.c_double(rho0), C.byref(th), C.byref(om))
        return th.value, om.value

    def plane_cp(self, side, p0, mach):
        """(x [M, D], C_P [M]) at the nodes of plane y index 0 (side 0) or N1 - 1 (side 1)."""
        n = C.c_int64()
        self._call("sllbm_plane_cp", C.c_int32(side), C.c_double(p0), C.c_double(mach), None, None, C.byref(n))
        x = np.zeros((n.value, self.D))
        cp = np.zeros(n.value)
        self._call("sllbm_plane_cp", C.c_int32(side), C.c_double(p0), C.c_double(mach), _ptr(x)[0], _ptr(cp)[0],
                   C.byref(n))
        return x, cp

    def mlp_path(self, path):
        """capi.MLP_TENSOR (tensor cores, default) or capi.MLP_SIMT (CUDA cores)."""
        self._call("sllbm_mlp_path", C.c_int32(path))

    def debug_wait_limit(self, log2_cycles):
        """Test hook: bound the tensor-core / bulk-copy waits by 2^log2_cycles
        SM cycles (0: the default, about a second)."""
        self._call("sllbm_debug_wait_limit", C.c_int32(log2_cycles))

    def device_status(self):
        """Synchronise and return (and clear) the context's device status word."""
        v = C.c_int32(0)
        self._call("sllbm_device_status", C.byref(v))
        return v.value

    # ---------------------------------------------------------------- readout
    def moments(self):
        rho = np.zeros(self.N)
        u = np.zeros((self.N, self.D))
        T = np.zeros(self.N)
        self._call("sllbm_read_moments", _ptr(rho)[0], _ptr(u)[0], _ptr(T)[0], 0)
        return rho, u, T

    def moments_into(self, rho, u, T):
        pr, dev = _ptr(rho)
        self._call("sllbm_read_moments", pr, _ptr(u)[0], _ptr(T)[0], dev)

    def conservation(self, check=True):
        out = np.zeros(self.D + 2)
        rc = capi.lib().sllbm_conservation(self.h, _ptr(out)[0])
        if check:
            capi.check(rc, self.h)
        return out, rc

    def departure_records(self):
        Q, N, D = self.Q, self.N, self.D
        r = dict(kind=np.zeros((Q, N), np.int32), src=np.zeros((Q, N), np.int32),
                 bid=np.zeros((Q, N), np.int32), cell=np.zeros((Q, N), np.int32),
                 xi=np.zeros((Q, N, D)), xsrc=np.zeros((Q, N, D)))
        self._call("sllbm_departure_records", *[_ptr(r[k])[0] for k in ("kind", "src", "bid", "cell", "xi", "xsrc")])
        return r
