"""The allocation-free spatial hash (sph_cell_sort_noalloc) against the substep's own hash.

Callers that cannot allocate device memory -- an engine plugin whose device memory belongs
to the engine's allocator, a haptic loop that must not allocate after start-up, or code
running under stream capture, where cudaMalloc is not allowed -- use this entry point; its
scratch is a fixed device array inside the library.  The result must equal, bit for bit,
the keys, stable order and cell ranges that sph_get_sort reports after the first substep of
the same particles.  Two calls in a row check that state kept in the shared scratch array
from one call does not leak into the next.  Collected last so that a run which stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2511_15908_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15908_gb300 import build, sph as _sph
    build.build()
    _sph.load()
    return _sph


def _reference(sph, sc):
    """Keys, order (as input indices = ids), cell_start from the substep's own hash, and the
    positions the first substep hashed (id order)."""
    sim = sph.Simulation(sc)
    x0 = sim.state()["x"]                     # positions before the first substep, id order
    sim.step(1)
    keys, ids, cs = sim.sort()
    sim.close()
    return x0, keys, ids, cs


@pytest.mark.parametrize("seeds", [(0, 1)])
def test_noalloc_sort_equals_substep_hash_twice(sph, seeds):
    import torch
    for seed in seeds:                         # two calls in a row
        sc = scenes.with_velocity_noise(scenes.dam_break(seed=seed), seed=seed, sigma=0.3)
        x0, keys, ids, cs = _reference(sph, sc)
        x4 = np.zeros((x0.shape[0], 4), np.float32)
        x4[:, :3] = x0
        xd = torch.tensor(x4, device="cuda")
        k, o, c = sph.cell_sort_noalloc(sc.params, xd)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(k.cpu().numpy().astype(np.uint32), keys)
        np.testing.assert_array_equal(o.cpu().numpy(), ids)
        np.testing.assert_array_equal(c.cpu().numpy().astype(np.uint32), cs)


def test_noalloc_rejects_sizes_beyond_the_limit(sph):
    import torch
    sc = scenes.dam_break(seed=0)
    x = torch.zeros((sph.NOALLOC_MAX_PARTICLES + 1, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(sph.SphError) as e:
        sph.cell_sort_noalloc(sc.params, x)
    assert e.value.status == sph.ERR_CAPACITY
    big = dict(sc.params, hi=(50.0, 50.0, 50.0))           # far more cells than the limit
    with pytest.raises(sph.SphError) as e:
        sph.cell_sort_noalloc(big, torch.zeros((16, 4), dtype=torch.float32, device="cuda"))
    assert e.value.status == sph.ERR_CAPACITY


def test_noalloc_cell_start_only_4_byte_aligned(sph):
    # a caller's cell_start that is only 4-byte aligned takes the scalar path of the scan
    import torch
    sc = scenes.with_velocity_noise(scenes.dam_break(seed=2), seed=2, sigma=0.3)
    x0, keys, ids, cs = _reference(sph, sc)
    x4 = np.zeros((x0.shape[0], 4), np.float32)
    x4[:, :3] = x0
    xd = torch.tensor(x4, device="cuda")
    n = x0.shape[0]
    buf = torch.zeros(cs.size + 1, dtype=torch.int32, device="cuda")
    assert (buf.data_ptr() + 4) % 16 != 0
    out = (torch.empty(n, dtype=torch.int32, device="cuda"),
           torch.empty(n, dtype=torch.int32, device="cuda"), buf[1:])
    k, o, c = sph.cell_sort_noalloc(sc.params, xd, out=out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(k.cpu().numpy().astype(np.uint32), keys)
    np.testing.assert_array_equal(o.cpu().numpy(), ids)
    np.testing.assert_array_equal(c.cpu().numpy().astype(np.uint32), cs)
