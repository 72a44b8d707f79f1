"""GPU parity of the tensor-memory row-tile kernel (SLLBM_STREAM_ROWS_TMEM,
k_step_rows_tmem) against the FP64 oracle.

The kernel takes tiles of 512 arrival nodes (whole periodic x rows: 2 x 2
rows of 128 nodes, 4 x 2 of 64, 4 x 4 of 32 in 3D; 2 .. 16 rows in 2D), keeps
the streamed state in tensor memory and stages the tile's source rows in
shared memory by bulk copies.  The cases cover each tile shape, a ragged last
y tile (idle rows), isothermal walls (bounce-back records with the thermal
correction), equilibrium boundaries (mixing layer) and the 2D set.
Tolerance: FP32-offset populations 1e-5 relative to each velocity's scale.
"""
import numpy as np
import pytest

from oracle import step as ost
from tests.oracle_cases import oracle_case
from workloads import get_config, initial_fields

pytestmark = pytest.mark.gpu

MODE = 7

CASES = {
    "channel_nx128": lambda: get_config("channel", cells=(64, 3, 3)),      # 128 x 7 x 6 nodes, ragged y tile
    "channel_nx64": lambda: get_config("channel", cells=(32, 3, 2)),       # 64 x 7 x 4
    "channel_nx32": lambda: get_config("channel", cells=(16, 4, 4)),       # 32 x 9 x 8, tiles of 4 x 4 rows
    "mixing_nx64": lambda: get_config("mixing", cells=(32, 4, 2)),         # equilibrium boundaries in y
    "box_d2q19_nx32": lambda: get_config("learned", cells=16),             # 2D, 16 rows per tile
    "box_d2q19_nx128": lambda: get_config("learned", cells=64),            # 2D, 4 rows per tile
}


def _scale_err(a, b, w):
    s = np.maximum(np.abs(b).max(axis=1, keepdims=True), np.asarray(w)[:, None])
    return float((np.abs(a - b) / s).max())


@pytest.mark.parametrize("name", list(CASES))
def test_rows_tmem_matches_oracle(built_lib, name):
    from paper_2412_09051_gb300.sim import Sim
    cfg = CASES[name]()
    mesh, xi, w, opp, par, rec = oracle_case(cfg)
    sim = Sim(cfg, precision="fp32", stream_mode=MODE)
    assert sim.info.stream_mode == MODE, "the row-tile kernel must be eligible for this mesh"
    rho, u, T = initial_fields(cfg, mesh.X)
    sim.init_state(rho, u, T)
    f, g = ost.init_equilibrium(rho, u, T, xi, w, par.cv)
    Tw = ost.isothermal_nodes(rec, par)
    worst = 0.0
    for k in range(3):
        f, g = ost.step(mesh, rec, f, g, xi, w, par, Tw=Tw)
        sim.step(1)
        assert sim.step_kernel() == "k_step_rows_tmem"
        fg, gg = sim.get_state()
        ef, eg = _scale_err(fg, f, w), _scale_err(gg, g, w)
        assert ef < 1e-5 and eg < 1e-5, (k, ef, eg)
        worst = max(worst, ef, eg)
    r0, u0, T0 = ost.moments(f, g, xi, par.cv)
    r1, u1, T1 = sim.moments()
    em = max(np.abs(r1 - r0).max(), np.abs(T1 - T0).max(), np.abs(u1 - u0).max() / max(1.0, np.abs(u0).max()))
    assert em < 1e-5
    assert sim.device_status() == 0
    print(f"PARITY rows_tmem {name} {mesh.N}: populations {worst:.2e} moments {em:.2e}")
    sim.close()


def test_rows_tmem_agrees_with_row_kernel(built_lib):
    """5 steps of the channel (128-node rows) against the one-block-per-row
    kernel: the same step up to FP32 summation order."""
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config("channel", cells=(64, 6, 4))
    a, b = Sim(cfg, stream_mode=MODE), Sim(cfg, stream_mode=8)
    X = a.node_coords()
    rho, u, T = initial_fields(cfg, X)
    for s in (a, b):
        s.init_state(rho, u, T)
        s.step(5)
    assert a.step_kernel() == "k_step_rows_tmem" and b.step_kernel() == "k_step_row_smem"
    fa, ga = a.get_state()
    fb, gb = b.get_state()
    _, w, _ = a.velocity_set()
    ef, eg = _scale_err(fa, fb, w), _scale_err(ga, gb, w)
    assert ef < 1e-5 and eg < 1e-5, (ef, eg)
    print(f"PARITY rows_tmem vs row_smem, 5 channel steps: {max(ef, eg):.2e}")
    a.close()
    b.close()


def test_row_tiles_are_the_default_for_d3q45(built_lib):
    """With the 45-velocity set, the automatic and the structured modes take
    the two-nodes-per-thread row-tile kernel on rows of 64 or 128 nodes, the
    one-node-per-thread row-tile kernel on rows of 32; SLLBM_STREAM_ROW_SMEM
    takes neither."""
    from paper_2412_09051_gb300.sim import Sim
    info = {"k_step_rows_pairs": 10, "k_step_rows_tmem": MODE, "k_step_row_smem": 2}
    for cells, mode, kernel in (((32, 3, 3), 0, "k_step_rows_pairs"), ((32, 3, 3), 2, "k_step_rows_pairs"),
                                ((64, 3, 3), 0, "k_step_rows_pairs"), ((16, 4, 4), 0, "k_step_rows_tmem"),
                                ((32, 3, 3), 7, "k_step_rows_tmem"), ((32, 3, 3), 8, "k_step_row_smem")):
        cfg = get_config("channel", cells=cells)
        s = Sim(cfg, stream_mode=mode)
        s.init_state(*initial_fields(cfg, s.node_coords()))
        s.step(1)
        assert s.step_kernel() == kernel, (cells, mode, s.step_kernel())
        assert s.info.stream_mode == info[kernel]
        s.close()


def test_rows_tmem_fullsize_channel_sampled(built_lib):
    """The benchmark's channel (128 x 97 x 96 nodes) in this mode: one step from
    the seeded state, sampled nodes (random, the first and last 40: both
    walls) computed by the oracle."""
    from oracle.departure import trace
    from oracle.mesh import Mesh
    from oracle.velocity_sets import velocity_set
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config("channel")
    m = cfg["mesh"]
    mesh = Mesh(m["kind"], m["p"], m["cells"], m["length"], m.get("stretch", 1.0), m.get("central", 0))
    xi, w, opp = velocity_set(cfg["velset"])
    par = ost.Params(cfg["dt"], cfg["gamma"], cfg["Pr"], cfg["mu_ref"], cfg["T_ref"], cfg["mu_exp"], cfg["bcs"])
    rho, u, T = initial_fields(cfg, mesh.X)
    rng = np.random.default_rng(12)
    nodes = np.unique(np.concatenate([rng.integers(0, mesh.n_nodes, 60), np.arange(40),
                                      mesh.n_nodes - 1 - np.arange(40)]))
    rec = trace(mesh, xi, opp, cfg["dt"], cfg["bcs"], nodes=nodes)
    f1, g1 = ost.step_sample_from_fields(mesh, rec, rho, u, T, xi, w, par)
    sim = Sim(cfg, stream_mode=MODE)
    assert sim.info.stream_mode == MODE
    sim.init_state(rho, u, T)
    sim.step(1)
    assert sim.step_kernel() == "k_step_rows_tmem"
    fg, gg = sim.get_state()
    worst = max(_scale_err(fg[:, nodes], f1, w), _scale_err(gg[:, nodes], g1, w))
    assert worst < 1e-5
    print(f"PARITY rows_tmem fullsize channel: {len(nodes)} sampled nodes, populations {worst:.2e}")
    sim.close()


TC_CASES = {
    "channel_nx128": lambda: get_config("channel", cells=(64, 3, 3)),      # isothermal walls, ragged y tile
    "mixing_nx128": lambda: get_config("mixing", cells=(64, 4, 3)),        # equilibrium boundaries
}


@pytest.mark.parametrize("name", list(TC_CASES))
def test_tensor_core_streaming_matches_oracle(built_lib, name):
    """SLLBM_STREAM_TENSOR: the (y, z) contraction of every velocity on the
    tensor cores (tcgen05 kind::tf32, operands split into TF32 hi and lo
    parts), the rest of the step as in the row-tile kernel; 3 steps against
    the oracle at the FP32 tolerance."""
    from paper_2412_09051_gb300.sim import Sim
    cfg = TC_CASES[name]()
    mesh, xi, w, opp, par, rec = oracle_case(cfg)
    sim = Sim(cfg, precision="fp32", stream_mode=9)
    assert sim.info.stream_mode == 9, "the tensor-core streaming must be eligible for this mesh"
    rho, u, T = initial_fields(cfg, mesh.X)
    sim.init_state(rho, u, T)
    f, g = ost.init_equilibrium(rho, u, T, xi, w, par.cv)
    Tw = ost.isothermal_nodes(rec, par)
    worst = 0.0
    for k in range(3):
        f, g = ost.step(mesh, rec, f, g, xi, w, par, Tw=Tw)
        sim.step(1)
        assert sim.step_kernel() == "k_step_rows_tmem_tc"
        fg, gg = sim.get_state()
        ef, eg = _scale_err(fg, f, w), _scale_err(gg, g, w)
        assert ef < 1e-5 and eg < 1e-5, (k, ef, eg)
        worst = max(worst, ef, eg)
    assert sim.device_status() == 0
    print(f"PARITY tensor-core streaming {name} {mesh.N}: populations {worst:.2e}")
    sim.close()


def test_tensor_core_streaming_fullsize_channel_sampled(built_lib):
    """The benchmark's channel with the tensor-core streaming: one step,
    sampled nodes computed by the oracle."""
    from oracle.departure import trace
    from oracle.mesh import Mesh
    from oracle.velocity_sets import velocity_set
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config("channel")
    m = cfg["mesh"]
    mesh = Mesh(m["kind"], m["p"], m["cells"], m["length"], m.get("stretch", 1.0), m.get("central", 0))
    xi, w, opp = velocity_set(cfg["velset"])
    par = ost.Params(cfg["dt"], cfg["gamma"], cfg["Pr"], cfg["mu_ref"], cfg["T_ref"], cfg["mu_exp"], cfg["bcs"])
    rho, u, T = initial_fields(cfg, mesh.X)
    rng = np.random.default_rng(13)
    nodes = np.unique(np.concatenate([rng.integers(0, mesh.n_nodes, 60), np.arange(40),
                                      mesh.n_nodes - 1 - np.arange(40)]))
    rec = trace(mesh, xi, opp, cfg["dt"], cfg["bcs"], nodes=nodes)
    f1, g1 = ost.step_sample_from_fields(mesh, rec, rho, u, T, xi, w, par)
    sim = Sim(cfg, stream_mode=9)
    sim.init_state(rho, u, T)
    sim.step(1)
    assert sim.step_kernel() == "k_step_rows_tmem_tc"
    fg, gg = sim.get_state()
    worst = max(_scale_err(fg[:, nodes], f1, w), _scale_err(gg[:, nodes], g1, w))
    assert worst < 1e-5
    print(f"PARITY tensor-core streaming fullsize channel: {len(nodes)} sampled nodes, populations {worst:.2e}")
    sim.close()


PAIR_CASES = {
    "channel_nx128": lambda: get_config("channel", cells=(64, 3, 3)),      # 2 x 2 rows of 128, ragged y tile
    "channel_nx64": lambda: get_config("channel", cells=(32, 3, 2)),       # 4 x 2 rows of 64
    "mixing_nx64": lambda: get_config("mixing", cells=(32, 4, 2)),         # equilibrium boundaries in y
    "mixing_nx128": lambda: get_config("mixing", cells=(64, 4, 3)),
    "box_d2q19_nx64": lambda: get_config("learned", cells=32),             # 2D, 8 rows per tile, periodic y
    "box_d2q19_nx128": lambda: get_config("learned", cells=64),            # 2D, 4 rows per tile
}


@pytest.mark.parametrize("name", list(PAIR_CASES))
def test_rows_pairs_matches_oracle(built_lib, name):
    """SLLBM_STREAM_ROWS_PAIRS: two arrival nodes per consumer thread, one
    TMA tensor copy per source population and velocity (bulk copies row by
    row across a periodic seam); 3 steps against the oracle at the FP32
    tolerance."""
    from paper_2412_09051_gb300.sim import Sim
    cfg = PAIR_CASES[name]()
    mesh, xi, w, opp, par, rec = oracle_case(cfg)
    sim = Sim(cfg, precision="fp32", stream_mode=10)
    assert sim.info.stream_mode == 10, "the two-nodes-per-thread kernel must be eligible for this mesh"
    rho, u, T = initial_fields(cfg, mesh.X)
    sim.init_state(rho, u, T)
    f, g = ost.init_equilibrium(rho, u, T, xi, w, par.cv)
    Tw = ost.isothermal_nodes(rec, par)
    worst = 0.0
    for k in range(3):
        f, g = ost.step(mesh, rec, f, g, xi, w, par, Tw=Tw)
        sim.step(1)
        assert sim.step_kernel() == "k_step_rows_pairs"
        fg, gg = sim.get_state()
        ef, eg = _scale_err(fg, f, w), _scale_err(gg, g, w)
        assert ef < 1e-5 and eg < 1e-5, (k, ef, eg)
        worst = max(worst, ef, eg)
    assert sim.device_status() == 0
    print(f"PARITY rows_pairs {name} {mesh.N}: populations {worst:.2e}")
    sim.close()


def test_rows_pairs_agrees_with_rows_tmem(built_lib):
    """5 channel steps against the one-node-per-thread row-tile kernel: the
    same step up to FP32 summation order."""
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config("channel", cells=(64, 6, 4))
    a, b = Sim(cfg, stream_mode=10), Sim(cfg, stream_mode=MODE)
    X = a.node_coords()
    rho, u, T = initial_fields(cfg, X)
    for s in (a, b):
        s.init_state(rho, u, T)
        s.step(5)
    assert a.step_kernel() == "k_step_rows_pairs" and b.step_kernel() == "k_step_rows_tmem"
    fa, ga = a.get_state()
    fb, gb = b.get_state()
    _, w, _ = a.velocity_set()
    ef, eg = _scale_err(fa, fb, w), _scale_err(ga, gb, w)
    assert ef < 1e-5 and eg < 1e-5, (ef, eg)
    assert a.device_status() == 0
    print(f"PARITY rows_pairs vs rows_tmem, 5 channel steps: {max(ef, eg):.2e}")
    a.close()
    b.close()


def test_rows_pairs_fullsize_channel_sampled(built_lib):
    """The benchmark's channel (128 x 97 x 96 nodes) with two nodes per
    thread: one step from the seeded state, sampled nodes (random, both
    walls) computed by the oracle."""
    from oracle.departure import trace
    from oracle.mesh import Mesh
    from oracle.velocity_sets import velocity_set
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config("channel")
    m = cfg["mesh"]
    mesh = Mesh(m["kind"], m["p"], m["cells"], m["length"], m.get("stretch", 1.0), m.get("central", 0))
    xi, w, opp = velocity_set(cfg["velset"])
    par = ost.Params(cfg["dt"], cfg["gamma"], cfg["Pr"], cfg["mu_ref"], cfg["T_ref"], cfg["mu_exp"], cfg["bcs"])
    rho, u, T = initial_fields(cfg, mesh.X)
    rng = np.random.default_rng(14)
    nodes = np.unique(np.concatenate([rng.integers(0, mesh.n_nodes, 60), np.arange(40),
                                      mesh.n_nodes - 1 - np.arange(40)]))
    rec = trace(mesh, xi, opp, cfg["dt"], cfg["bcs"], nodes=nodes)
    f1, g1 = ost.step_sample_from_fields(mesh, rec, rho, u, T, xi, w, par)
    sim = Sim(cfg, stream_mode=10)
    assert sim.info.stream_mode == 10
    sim.init_state(rho, u, T)
    sim.step(1)
    assert sim.step_kernel() == "k_step_rows_pairs"
    fg, gg = sim.get_state()
    worst = max(_scale_err(fg[:, nodes], f1, w), _scale_err(gg[:, nodes], g1, w))
    assert worst < 1e-5
    print(f"PARITY rows_pairs fullsize channel: {len(nodes)} sampled nodes, populations {worst:.2e}")
    sim.close()


PAIR4_CASES = {
    "channel_p4_nx128": lambda: get_config("channel", cells=(32, 3, 3), p=4),   # 4 x 1 rows of 128, ragged y tile
    "channel_p4_nx64": lambda: get_config("channel", cells=(16, 3, 3), p=4),    # 8 x 1 rows of 64, ragged y tile
}


@pytest.mark.parametrize("name", list(PAIR4_CASES))
def test_rows_pairs_order4_matches_oracle(built_lib, name):
    """The two-nodes-per-thread row tiles at the paper's order p = 4 (25
    (y, z) taps, nine x taps per node over ten row sums, two pair classes):
    3 steps against the oracle at the FP32 tolerance."""
    from paper_2412_09051_gb300.sim import Sim
    cfg = PAIR4_CASES[name]()
    mesh, xi, w, opp, par, rec = oracle_case(cfg)
    sim = Sim(cfg, precision="fp32", stream_mode=10)
    assert sim.info.stream_mode == 10, "the order-4 row tiles must be eligible for this mesh"
    rho, u, T = initial_fields(cfg, mesh.X)
    sim.init_state(rho, u, T)
    f, g = ost.init_equilibrium(rho, u, T, xi, w, par.cv)
    Tw = ost.isothermal_nodes(rec, par)
    worst = 0.0
    for k in range(3):
        f, g = ost.step(mesh, rec, f, g, xi, w, par, Tw=Tw)
        sim.step(1)
        assert sim.step_kernel() == "k_step_rows_pairs"
        fg, gg = sim.get_state()
        ef, eg = _scale_err(fg, f, w), _scale_err(gg, g, w)
        assert ef < 1e-5 and eg < 1e-5, (k, ef, eg)
        worst = max(worst, ef, eg)
    assert sim.device_status() == 0
    print(f"PARITY rows_pairs order 4 {name} {mesh.N}: populations {worst:.2e}")
    sim.close()


def test_rows_pairs_order4_agrees_with_row_kernel(built_lib):
    """5 steps of the order-4 channel (128-node rows) against the order-4
    one-block-per-row kernel: the same step up to FP32 summation order."""
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config("channel", cells=(32, 4, 3), p=4)
    a, b = Sim(cfg, stream_mode=10), Sim(cfg, stream_mode=8)
    X = a.node_coords()
    rho, u, T = initial_fields(cfg, X)
    for s in (a, b):
        s.init_state(rho, u, T)
        s.step(5)
    assert a.step_kernel() == "k_step_rows_pairs" and b.step_kernel() == "k_step_row_p"
    fa, ga = a.get_state()
    fb, gb = b.get_state()
    _, w, _ = a.velocity_set()
    ef, eg = _scale_err(fa, fb, w), _scale_err(ga, gb, w)
    assert ef < 1e-5 and eg < 1e-5, (ef, eg)
    print(f"PARITY rows_pairs order 4 vs row kernel, 5 channel steps: {max(ef, eg):.2e}")
    a.close()
    b.close()
