"""A caller's device allocator (sllbm_set_allocator): the context's buffers
come from PyTorch's caching allocator, the step is bit-identical to a
context with its own buffers, everything goes back at sllbm_destroy, and
memory the library cannot use is refused."""
import numpy as np
import pytest

from workloads import get_config, initial_fields

pytestmark = pytest.mark.gpu


def _run(cfg, X, steps=3):
    from paper_2412_09051_gb300.sim import Sim
    s = Sim(cfg)
    s.init_state(*initial_fields(cfg, X))
    s.step(steps)
    return s


@pytest.mark.parametrize("cells", [(4, 6, 3), (32, 3, 2)])
def test_torch_allocator_serves_every_buffer(built_lib, cells):
    import torch
    from paper_2412_09051_gb300 import capi
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config("channel", cells=cells)
    ref = Sim(cfg)
    X = ref.node_coords()
    ref.close()
    ref = _run(cfg, X)
    alloc = capi.TorchAllocator()
    before = torch.cuda.memory_allocated()
    with alloc:
        s = _run(cfg, X)
    held = sum(t.numel() for t in alloc.blocks.values())
    assert held >= 2 * s.info.state_bytes                       # both population buffers and more
    assert torch.cuda.memory_allocated() - before >= held
    assert np.array_equal(s.get_state_raw(), ref.get_state_raw())
    assert s.step_kernel() == ref.step_kernel()
    s.close()
    assert not alloc.blocks                                      # everything handed back
    ref.close()


def test_unusable_memory_is_refused(built_lib):
    """Memory that is not 256-byte aligned: the create fails with an argument
    error and every block it took is handed back; an allocator that returns
    NULL gives SLLBM_ERR_NOMEM."""
    import ctypes as C
    import torch
    from paper_2412_09051_gb300 import capi
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config("tgv2d", cells=4)
    blocks = {}

    def take(nbytes, user):
        t = torch.empty(int(nbytes) + 512, dtype=torch.uint8, device="cuda:0")
        p = t.data_ptr() + 16
        blocks[p] = t
        return p

    def give(ptr, user):
        blocks.pop(ptr, None)

    fa, ff = capi.ALLOC_FN(take), capi.FREE_FN(give)
    L = capi.lib()
    assert L.sllbm_set_allocator(fa, ff, None) == 0
    try:
        with pytest.raises(capi.SllbmError) as e:
            Sim(cfg)
        assert e.value.code == -1 and "256-byte" in str(e.value)
        assert not blocks
        fn = capi.ALLOC_FN(lambda n, u: None)
        assert L.sllbm_set_allocator(fn, ff, None) == 0
        with pytest.raises(capi.SllbmError) as e:
            Sim(cfg)
        assert e.value.code == -4
    finally:
        assert L.sllbm_set_allocator(capi.ALLOC_FN(), capi.FREE_FN(), None) == 0
    # the default allocator again
    s = Sim(cfg)
    s.close()
