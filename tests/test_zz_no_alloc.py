"""The allocation-free spatial hash (sph_cell_sort_noalloc) against the substep's own hash
and the oracle's hash and counting sort.

Callers that cannot allocate device memory -- an engine plugin whose device memory belongs
to the engine's allocator, a haptic loop that must not allocate after start-up, or code
running under stream capture, where cudaMalloc is not allowed -- use this entry point; its
scratch is a fixed device array inside the library.  The result must equal, bit for bit,
the keys, stable order and cell ranges that sph_get_sort reports after the first substep of
the same particles.  Two calls in a row check that state kept in the shared scratch array
from one call does not leak into the next.  Collected last so that a run which stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
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
        # and the oracle's FP32 hash and stable counting sort of the same positions
        k_orc, _ = oracle.hash_keys(sc.params, x0)
        cs_orc, src = oracle.counting_sort(k_orc, int(cs.size) - 1)
        np.testing.assert_array_equal(k.cpu().numpy().astype(np.uint32), k_orc[src])
        np.testing.assert_array_equal(o.cpu().numpy(), src)
        np.testing.assert_array_equal(c.cpu().numpy().astype(np.uint32), cs_orc)


def test_noalloc_rejects_sizes_beyond_the_limit(sph):
    import torch
    sc = scenes.dam_break(seed=0)
    L = sph.load()
    P = sph.make_params(sc.params, 1.0)
    tiny = [torch.zeros(16, dtype=torch.int32, device="cuda") for _ in range(3)]
    x = torch.zeros((16, 4), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    # the library itself refuses before touching any buffer: too many particles ...
    r = L.sph_cell_sort_noalloc(ctypes.byref(P), x.data_ptr(), sph.NOALLOC_MAX_PARTICLES + 1,
                                tiny[0].data_ptr(), tiny[1].data_ptr(), tiny[2].data_ptr(), st)
    assert r == sph.ERR_CAPACITY
    # ... far more cells than the limit, and a cell count beyond the range of int
    for hi in ((50.0, 50.0, 50.0), (3.0e38, 1.0, 1.0)):
        Pb = sph.make_params(dict(sc.params, hi=hi), 1.0)
        r = L.sph_cell_sort_noalloc(ctypes.byref(Pb), x.data_ptr(), 16, tiny[0].data_ptr(),
                                    tiny[1].data_ptr(), tiny[2].data_ptr(), st)
        assert r == sph.ERR_CAPACITY
    torch.cuda.synchronize()
    # the binding refuses the same sizes before it allocates the outputs
    with pytest.raises(sph.SphError) as e:
        sph.cell_sort_noalloc(dict(sc.params, hi=(50.0, 50.0, 50.0)), x)
    assert e.value.status == sph.ERR_CAPACITY


def test_noalloc_overfull_cell_is_a_permutation_with_ascending_keys(sph):
    # 600 particles in one cell (more than the 512 the stable in-cell rank handles) plus a
    # sparse set elsewhere: the over-full cell's members come in some order, every other
    # cell keeps input order, keys ascend and cell_start matches them
    import torch
    rng = np.random.default_rng(5)
    p = scenes.make_params(0.02, 1e-3, (-0.1, -0.1, -0.1), (0.1, 0.1, 0.1))
    packed = 0.0301 + rng.uniform(0.0, 0.005, (600, 3))
    loose = rng.uniform(-0.09, 0.09, (400, 3))
    x0 = np.concatenate([loose[:200], packed, loose[200:]]).astype(np.float32)
    x4 = np.zeros((x0.shape[0], 4), np.float32)
    x4[:, :3] = x0
    k, o, c = sph.cell_sort_noalloc(p, torch.tensor(x4, device="cuda"))
    torch.cuda.synchronize()
    k, o, c = k.cpu().numpy().astype(np.int64), o.cpu().numpy(), c.cpu().numpy().astype(np.int64)
    assert np.all(np.diff(k) >= 0)
    assert np.array_equal(np.sort(o), np.arange(x0.shape[0]))
    np.testing.assert_array_equal(c, np.searchsorted(k, np.arange(c.size)))
    k_orc, _ = oracle.hash_keys(p, x0)
    np.testing.assert_array_equal(k, k_orc[o])
    full = np.bincount(k, minlength=c.size - 1)
    other = full[k] <= 512
    same = (k[1:] == k[:-1]) & other[1:]
    assert np.all(o[1:][same] > o[:-1][same]), "ties out of input order in a cell of <= 512"


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
