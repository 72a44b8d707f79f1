"""Benchmark of the fused SLLBM step (MLUPS and HBM roofline fraction).

Default workload: the 3D supersonic channel, 64 x 48 x 48 order-2 cells
(128 x 97 x 96 = 1,191,936 nodes), D3Q45, FP32-offset storage, structured
streaming; one step = one launch of the fused stream + collide kernel over
all nodes.  The populations (2 x 45 x 4 B x N per buffer, 429 MB) exceed the
129 MB L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--config NAME] [--impl reference]
Under torchrun each rank runs an independent replica on its own GPU (the
method does not exchange data between replicas); value sums all ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        cmd = ["nvidia-smi", "-i", str(self.index),
               "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
               "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
               "clocks_event_reasons.sw_power_cap,clocks.mem,clocks.max.mem,power.draw",
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 6:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def col(k):
            out = []
            for r in self.rows:
                if len(r) > k:
                    try:
                        out.append(float(r[k]))
                    except ValueError:
                        pass
            return out
        sm, mx, mem, mmx, pw = col(0), col(1), col(6), col(7), col(8)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[2 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "mem_mhz": statistics.median(mem) if mem else None, "mem_max_mhz": max(mmx) if mmx else None,
                "power_w_max": max(pw) if pw else None, "reasons": reasons, "samples": len(self.rows)}


def aggregate(ms_total, nodes, steps, e2e_s, dist=None, device="cpu"):
    """Whole-job numbers over the replicas: the slowest rank's time (max over
    ranks) and all ranks' nodes (sum).  Returns (ms_max, nodes_total,
    MLUPS, e2e MLUPS)."""
    import torch
    t = torch.tensor([float(ms_total), float(e2e_s)], dtype=torch.float64, device=device)
    n = torch.tensor([float(nodes)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
    ms_max, e2e_max = (float(v) for v in t.tolist())
    total = float(n.item())
    return ms_max, total, total * steps / (ms_max / 1e3) / 1e6, total / e2e_max / 1e6


def workload_config(cfg, ws=1):
    """The `config` object of the JSON line (shared by both arms)."""
    m = cfg["mesh"]
    periodic = {0: (1, 1, 1), 1: (1, 0, 1), 2: (1, 0, 1), 3: (1, 0)}[m["kind"]]
    N = 1
    for d, c in enumerate(m["cells"]):
        N *= c * m["p"] + (0 if periodic[d] else 1)
    Q = {"D2Q9": 9, "D2Q19": 19, "D2Q25": 25, "D3Q45": 45}[cfg["velset"]]
    rb = 8 if cfg.get("precision") == "fp64" else 4
    return {"workload": f"{cfg['name']} ({cfg['velset']}, {'FP32-offset' if rb == 4 else 'FP64'}, "
                        f"{'gather' if m['kind'] == 3 else 'structured'} streaming)",
            "nodes": N, "Q": Q, "replicas": ws,
            "l2": (f"inputs larger than L2: state {2 * Q * N * rb / 1e6:.0f} MB per buffer pair"
                   if 2 * Q * N * rb > 129e6 else
                   f"inputs smaller than L2 ({2 * Q * N * rb / 1e6:.0f} MB per buffer pair): no flush, L2-warm")}


def algorithmic_bytes_per_node(Q, real_bytes):
    """Every population of f and g read once and written once."""
    return 2 * 2 * Q * real_bytes


# ------------------------------------------------------------------ oracle arm
def oracle_sample_rate(cfg_name, target_s=10.0, cores=1, seed=0):
    """Oracle (FP64 numpy) MLUPS on a bounded sample of arrival nodes of the
    workload: one step (stream, thermal correction, collision) for M nodes,
    departure tracing excluded (setup).  Runs in this process."""
    import numpy as np
    from oracle import step as ost
    from oracle.departure import trace
    from oracle.mesh import Mesh
    from oracle.velocity_sets import velocity_set
    from workloads import get_config, initial_fields
    cfg = get_config(cfg_name)
    m = cfg["mesh"]
    mesh = Mesh(m["kind"], m["p"], m["cells"], m["length"], m.get("stretch", 1.0), m.get("central", 0),
                m.get("thickness", 0.12))
    xi, w, opp = velocity_set(cfg["velset"])
    par = ost.Params(cfg["dt"], cfg["gamma"], cfg["Pr"], cfg["mu_ref"], cfg["T_ref"], cfg["mu_exp"], cfg["bcs"])
    rho, u, T = initial_fields(cfg, mesh.X)
    rng = np.random.default_rng(seed)
    M = 256
    total_nodes, total_t = 0, 0.0
    while total_t < target_s:
        nodes = np.unique(rng.integers(0, mesh.n_nodes, M))
        rec = trace(mesh, xi, opp, cfg["dt"], cfg["bcs"], nodes=nodes)
        need = rec["kind"] != 0
        cells = np.unique(rec["cell"][rec["cell"] >= 0])
        sup = np.unique(mesh.cell_nodes(cells).ravel())
        f = np.zeros((len(xi), mesh.n_nodes))
        g = np.zeros((len(xi), mesh.n_nodes))
        f[:, sup], g[:, sup] = ost.init_equilibrium(rho[sup], u[sup], T[sup], xi, w, par.cv)
        Tw = ost.isothermal_nodes(rec, par)
        t0 = time.perf_counter()
        fs, gs = ost.stream(mesh, rec, f, g, xi, w, par)
        fs, gs = ost.thermal_correction(fs, gs, xi, w, par, Tw)
        ost.collide(fs, gs, xi, w, par)
        dt = time.perf_counter() - t0
        total_nodes += len(nodes)
        total_t += dt
        M = min(200000, M * 2)
    return {"value": total_nodes / total_t / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{total_nodes} random arrival nodes of {cfg['name']}, one step each "
                      f"(stream + thermal correction + collision, FP64 numpy), {total_t:.1f} s"}


def mlp_flops_per_node(Q, H=64):
    """Flops of the learned correction's network per node (Q -> H -> H -> Q),
    2 per multiply-add; the moment transform and projection not counted."""
    return 2 * (Q * H + H * H + H * Q)


def _cfg_of(args):
    from workloads import get_config
    over = {}
    if args.cells:
        over["cells"] = tuple(int(c) for c in args.cells.split(","))
    if args.p:
        over["p"] = args.p
    return get_config(args.config, **over)


def run_oracle_subprocess(cfg_name, target_s, all_cores=False):
    """The oracle on one host core (a single-threaded subprocess); with
    all_cores, also one such process per host core (up to 16) run at once on
    different node samples, their rates summed."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")

    def launch(seed):
        code = ("import json,sys; sys.path.insert(0, %r); import bench; "
                "print(json.dumps(bench.oracle_sample_rate(%r, %r, 1, %d)))" % (ROOT, cfg_name, target_s, seed))
        return subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                text=True, env=env, cwd=ROOT)

    def result(pr):
        out, err = pr.communicate()
        if pr.returncode != 0:
            return None, err[-300:]
        return json.loads(out.strip().splitlines()[-1]), ""

    one, err = result(launch(0))
    if one is None:
        return {"value": None, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": "failed: " + err}
    if all_cores:
        n = max(1, min(16, os.cpu_count() or 1))
        rs = [result(p) for p in [launch(1 + k) for k in range(n)]]
        vals = [r[0]["value"] for r in rs if r[0] is not None]
        if len(vals) == n:
            one["all_cores"] = {"value": sum(vals), "unit": "MLUPS", "cores": n,
                                "sample": f"{n} single-threaded oracle processes at once, each on its own seeded "
                                          f"sample of about {target_s:.0f} s; rates summed"}
    return one


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, ws, rank, local):
    import numpy as np
    import torch
    from paper_2412_09051_gb300.sim import Sim
    from workloads import get_config, initial_fields
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cfg = _cfg_of(args)
    stream = torch.cuda.Stream()
    sim = Sim(cfg, device=local, stream=stream.cuda_stream, stream_mode=args.mode)
    N, Q = sim.N, sim.Q
    X = sim.node_coords()
    rho, u, T = initial_fields(cfg, X)
    sim.init_state(rho, u, T)
    real_bytes = 8 if sim.fp64 else 4
    if args.learned != "none":
        # the learned collision correction with a seeded random network of the
        # trained shape (timing does not depend on the weights' values)
        from paper_2412_09051_gb300 import capi
        from paper_2412_09051_gb300.learned import init_params, install_params
        install_params(sim, init_params(Q, 0), np.ones(Q, np.float32), 1e-3)
        sim.mlp_path(capi.MLP_TENSOR if args.learned == "tensor" else capi.MLP_SIMT)
    # warm-up
    sim.step(args.warmup)
    sim.sync()
    cons0, _ = sim.conservation(check=False)     # FP64 sums before the timed steps (untimed)
    # `repeats` timing windows of K steps each, every window bracketed by a
    # barrier and a device synchronisation; the reported window is the median
    # one (best and all windows are reported beside it)
    windows, per = [], []
    with ClockSampler(local) as clk:
        for rep in range(args.repeats):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                ev[0].record(stream)
                for k in range(args.steps):
                    sim.step(1)
                    ev[k + 1].record(stream)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            per += [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
            windows.append(ev[0].elapsed_time(ev[-1]))
    ms_total = statistics.median(windows)
    cons, rc = sim.conservation(check=False)
    kernel_name = sim.step_kernel()
    dev_status = sim.device_status() if args.learned != "none" else 0

    # end to end through the C ABI: every step, the H2D copy of the step's
    # input state from pinned host memory, its upload into the context
    # (sllbm_set_state_raw from device memory), one step and the D2H read of
    # the moments into pinned host memory.  The H2D copies run one step ahead
    # on their own stream into two staging buffers, so step k's copy-in
    # overlaps step k-1's compute and copy-out; the bytes per step are unchanged.
    dt_ = torch.float32 if real_bytes == 4 else torch.float64
    raw = torch.empty((Q, N, 2), dtype=dt_).pin_memory()
    sim.get_state_raw(raw)
    sim.sync()
    mr = torch.empty(N, dtype=torch.float64).pin_memory()
    mu_ = torch.empty((N, sim.D), dtype=torch.float64).pin_memory()
    mT = torch.empty(N, dtype=torch.float64).pin_memory()
    stage = [torch.empty((Q, N, 2), dtype=dt_, device=f"cuda:{local}") for _ in range(2)]
    cs = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    ke = max(3, min(args.steps, 10))

    def upload(k):
        b = k % 2
        if k >= 2:
            cs.wait_event(consumed[b])          # the context has taken the buffer's previous contents
        with torch.cuda.stream(cs):
            stage[b].copy_(raw, non_blocking=True)
            copied[b].record(cs)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    upload(0)
    for k in range(ke):
        if k + 1 < ke:
            upload(k + 1)
        b = k % 2
        stream.wait_event(copied[b])
        sim.set_state_raw(stage[b])
        consumed[b].record(stream)
        sim.step(1)
        sim.moments_into(mr, mu_, mT)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / ke
    del stage
    h2d = 2 * Q * N * real_bytes
    d2h = N * (sim.D + 2) * 8

    ms_max, total_nodes, value, e2e_value = aggregate(ms_total, N, args.steps, e2e_s, dist, "cuda")
    mlups_rank = N * args.steps / (ms_total / 1e3) / 1e6
    avg_launch_ms = statistics.mean(per)
    peaks, psrc = _peaks()
    alg_bytes = algorithmic_bytes_per_node(Q, real_bytes) * N
    achieved = alg_bytes / (avg_launch_ms / 1e3) / 1e9
    # curved meshes stream a per-(node, velocity) departure table (cell code
    # + D reference coordinates) besides the populations: second roofline
    table_bytes = sim.info.table_bytes if "gather" in kernel_name else 0
    line = None
    if rank == 0:
        traffic = None
        tf = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tf):
            try:
                # DRAM bytes per launch from one ncu capture, keyed by workload and kernel
                traffic = json.load(open(tf)).get(f"{cfg['name']}|{kernel_name}")
            except Exception:
                traffic = None
        line = {
            "metric": "MLUPS (node updates/s, all Q of f and g)",
            "value": round(value, 2),
            "unit": "MLUPS",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(ms_max / args.steps, 5),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32" if real_bytes == 4 else "f64",
            "data": "synthetic (seeded laminar profile + 10% Philox perturbation)" if args.config == "channel"
                    else "synthetic (seeded)",
            "config": workload_config(cfg, ws),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                         "peak_source": f"{psrc} (copy bandwidth)",
                         "algorithmic_bytes_per_launch": alg_bytes,
                         **({"with_table": {"algorithmic_bytes_per_launch": alg_bytes + table_bytes,
                                            "achieved": round((alg_bytes + table_bytes) / (avg_launch_ms / 1e3) / 1e9, 1),
                                            "frac": round((alg_bytes + table_bytes) / (avg_launch_ms / 1e3) / 1e9
                                                          / peaks["hbm_gbs"], 4)}} if table_bytes else {}),
                         "kernel": kernel_name + f"<{cfg['velset']}>" +
                                   ("" if args.learned == "none" else
                                    f" (learned, MLP on {'tensor' if args.learned == 'tensor' else 'CUDA'} cores)")},
            "e2e": {"value": round(e2e_value, 2), "unit": "MLUPS", "h2d_bytes_per_step": h2d * ws,
                    "d2h_bytes_per_step": d2h * ws},
            "gpu_launches": args.steps * args.repeats,
            "repeats": {"n": args.repeats, "steps_each": args.steps,
                        "median_mlups": round(N * args.steps / (statistics.median(windows) / 1e3) / 1e6, 2),
                        "best_mlups": round(N * args.steps / (min(windows) / 1e3) / 1e6, 2),
                        "window_ms": [round(w, 4) for w in windows],
                        "note": "value is the median window; gpu_launches counts every window"},
            "clocks": clk.summary(),
            "conservation_rc": rc,
            # relative change over the timed steps of the FP64 sums of rho and of
            # 2 rho E: interpolation on a non-uniform mesh and at the walls'
            # reflected departure points is not conservative, isothermal walls
            # exchange energy, open boundaries both
            "conservation_drift": {"mass": float((cons[0] - cons0[0]) / cons0[0]),
                                   "energy": float((cons[-1] - cons0[-1]) / cons0[-1]), "steps": args.steps},
            **({"learned": {"mlp": args.learned, "device_status": dev_status,
                            "mlp_tflops": round(mlp_flops_per_node(Q) * N / (avg_launch_ms / 1e3) / 1e12, 2)}}
               if args.learned != "none" else {}),
            "per_rank_mlups": round(mlups_rank, 2),
        }
    sim.close()
    if dist:
        dist.destroy_process_group()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--repeats", type=int, default=3, help="timed windows of --steps steps; value is the median")
    ap.add_argument("--config", default="channel")
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cells", default=None, help="override the cell counts, e.g. 32,48,24 (profiling runs)")
    ap.add_argument("--p", type=int, default=None, help="override the Lagrange order (e.g. 4, the paper's)")
    ap.add_argument("--mode", type=int, default=0, help="streaming mode (include/sllbm.h SLLBM_STREAM_*)")
    ap.add_argument("--learned", default="none", choices=["none", "tensor", "simt"],
                    help="time the learned-correction step (config learned): MLP on tensor or CUDA cores")
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        if rank != 0:
            return 0
        cb = run_oracle_subprocess(args.config, max(5.0, args.cpu_seconds * args.steps / max(args.steps, 1)))
        line = {"impl": "reference", "metric": "MLUPS (node updates/s, all Q of f and g)", "value": cb["value"],
                "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded)", "config": workload_config(_cfg_of(args)),
                "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                                            "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0
    from paper_2412_09051_gb300 import build as b
    if rank == 0:
        b.build()
    line = run_gpu(args, ws, rank, local)
    if rank == 0:
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = run_oracle_subprocess(args.config, args.cpu_seconds, all_cores=True)
        print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
