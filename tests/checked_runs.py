"""Small step runs of every kernel family on one library, saved to an .npz.

A process loads one libsllbm, so tests/test_gpu_checked.py runs these cases on
the bounds-checked debug build (libsllbm_checked.so) in a child process and on
the release build in the test process, and compares the two.
Usage: python -m tests.checked_runs OUT.npz [LIBRARY]
"""
import sys

import numpy as np

from tests.oracle_cases import box_cfg
from workloads import get_config, initial_fields

STEPS = 3


def cases():
    """[(key, cfg, precision, stream_mode, learned path or None)]: the parity
    cases in every streaming mode (curved meshes: the gather modes), the
    order-4 warp tiles and rows, the smallest meshes, and the learned step on
    the tensor and CUDA cores."""
    from tests.test_gpu_parity import CASES, _cfg
    out = []
    for name in CASES:
        cfg, prec = _cfg(name)
        for mode in (0, 1, 3, 4, 5, 6):
            if mode not in (0, 5) and cfg["mesh"]["kind"] == 3:
                continue
            out.append((f"{name}_m{mode}", cfg, prec, mode, None))
    for name, cells in (("channel", (4, 3, 3)), ("mixing", (4, 4, 3)), ("channel", (8, 3, 3))):
        out.append((f"{name}_p4_{cells[0]}x{cells[1]}x{cells[2]}_m2", get_config(name, cells=cells, p=4),
                    "fp32", 2, None))
    for velset, cells in (("D2Q19", (1, 1)), ("D2Q19", (2, 1)), ("D3Q45", (1, 1, 1))):
        cfg = box_cfg(cells=cells, p=2, L=(1.0,) * len(cells), dt=0.01, velset=velset)
        for prec in ("fp32", "fp64"):
            out.append((f"box_{velset}_{'x'.join(map(str, cells))}_{prec}", cfg, prec, 0, None))
    # the tensor-memory row-tile kernel on each tile shape
    from tests.test_gpu_rows_tmem import CASES as TM_CASES
    for name, mk in TM_CASES.items():
        out.append((f"rows_tmem_{name}_m7", mk(), "fp32", 7, None))
    from tests.test_gpu_rows_tmem import PAIR_CASES
    for name, mk in PAIR_CASES.items():
        out.append((f"rows_pairs_{name}_m10", mk(), "fp32", 10, None))
    learned = get_config("learned", cells=8)
    learned["init"] = dict(kind="isentropic_vortex", mach=0.6, seed=3)
    for path in ("tensor", "simt"):
        out.append((f"learned_{path}", learned, "fp32", 0, path))
    return out


def keys():
    return [c[0] for c in cases()]


def run(out_path, lib_path=None):
    from paper_2412_09051_gb300 import capi
    from paper_2412_09051_gb300.sim import Sim
    L = capi.lib(lib_path)
    res = {"build_flags": np.int64(L.sllbm_build_flags())}
    for key, cfg, prec, mode, path in cases():
        s = Sim(cfg, precision=prec, stream_mode=mode)
        if path is not None:
            from tests.test_gpu_learned import _random_install
            _random_install(s, s.Q, seed=11, sigma=3e-2)
            s.mlp_path(capi.MLP_TENSOR if path == "tensor" else capi.MLP_SIMT)
        s.init_state(*initial_fields(cfg, s.node_coords()))
        s.step(STEPS)
        f, g = s.get_state()
        res[key + ".f"] = f
        res[key + ".g"] = g
        res[key + ".status"] = np.int64(s.device_status())
        res[key + ".kernel"] = np.array(s.step_kernel())
        s.close()
    np.savez(out_path, **res)


if __name__ == "__main__":
    run(sys.argv[1], sys.argv[2] if len(sys.argv) > 2 else None)
