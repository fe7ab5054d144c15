"""Pins of the FP64 surrogate oracle: library routines (torch float64, torch bf16
conversion), finite differences, and hand-placed descriptor cases (no GPU)."""
import numpy as np
import pytest
import torch

from oracle import mlp
from paper_2511_15908_gb300 import scenes


def _torch_mlp(params, norm, X):
    p = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    sizes = [(128, 269), (128,), (128, 128), (128,), (128, 128), (128,), (6, 128), (6,)]
    chunks, o = [], 0
    for s in sizes:
        n = int(np.prod(s))
        chunks.append(p[o:o + n].reshape(s))
        o += n
    xn = (torch.tensor(X, dtype=torch.float64) - torch.tensor(norm[:269], dtype=torch.float64)) \
        / torch.tensor(norm[269:538], dtype=torch.float64)
    h = xn
    for l in range(3):
        h = torch.nn.functional.gelu(torch.nn.functional.linear(h, chunks[2 * l], chunks[2 * l + 1]),
                                     approximate="tanh")
    y = torch.nn.functional.linear(h, chunks[6], chunks[7])
    return p, y


def _data(B=7, seed=0):
    rng = np.random.default_rng(seed)
    params = scenes.mlp_init_params(seed)
    params[128 * 269:128 * 269 + 128] = rng.normal(0, 0.1, 128)     # non-zero biases
    norm = np.concatenate([rng.normal(0, 1, 269), rng.uniform(0.5, 2, 269), rng.normal(0, 1, 6),
                           rng.uniform(0.5, 2, 6)]).astype(np.float32)
    X = rng.normal(0, 1.5, (B, 269)).astype(np.float32)
    T = rng.normal(0, 1, (B, 6)).astype(np.float32)
    return params, norm, X, T


def test_gelu_matches_torch_tanh_form():
    z = np.linspace(-6, 6, 241)
    ref = torch.nn.functional.gelu(torch.tensor(z, dtype=torch.float64), approximate="tanh").numpy()
    got = np.array([mlp.gelu(v) for v in z])
    np.testing.assert_allclose(got, ref, rtol=1e-14, atol=1e-15)
    d = 1e-6
    fd = np.array([(mlp.gelu(v + d) - mlp.gelu(v - d)) / (2 * d) for v in z])
    np.testing.assert_allclose([mlp.gelu_grad(v) for v in z], fd, rtol=1e-7, atol=1e-9)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(0, 10, 2000), [1.00390625, 1.01171875, -3.0078125, 0.0]]).astype(np.float32)
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([mlp.bf16(v) for v in x], np.float32)
    np.testing.assert_array_equal(got, ref)


def test_forward_and_gradient_match_torch_float64():
    params, norm, X, T = _data()
    p, y = _torch_mlp(params, norm, X)
    y_phys = y * torch.tensor(norm[544:550], dtype=torch.float64) + torch.tensor(norm[538:544], dtype=torch.float64)
    np.testing.assert_allclose(mlp.forward(params, norm, X, bf=False), y_phys.detach().numpy(), rtol=1e-12, atol=1e-12)
    tn = (torch.tensor(T, dtype=torch.float64) - torch.tensor(norm[538:544], dtype=torch.float64)) \
        / torch.tensor(norm[544:550], dtype=torch.float64)
    loss_t = ((y - tn) ** 2).mean()
    loss_t.backward()
    loss, G = mlp.grad(params, norm, X, T, bf=False)
    assert loss == pytest.approx(loss_t.item(), rel=1e-12)
    np.testing.assert_allclose(G, p.grad.numpy(), rtol=1e-9, atol=1e-12)


def test_gradient_matches_finite_differences():
    params, norm, X, T = _data(B=3, seed=2)
    _, G = mlp.grad(params, norm, X, T, bf=False)
    rng = np.random.default_rng(3)
    for idx in rng.choice(params.size, 12, replace=False):
        # perturb in float64 by evaluating the oracle at +-d (params are FP32: use a step
        # large enough to be exact in FP32 and check to the FP32-induced accuracy)
        d = 1e-3 * max(1.0, abs(float(params[idx])))
        pp, pm = params.copy(), params.copy()
        pp[idx] += np.float32(d)
        pm[idx] -= np.float32(d)
        dd = float(pp[idx]) - float(pm[idx])
        lp, _ = mlp.grad(pp, norm, X, T, bf=False)
        lm, _ = mlp.grad(pm, norm, X, T, bf=False)
        fd = (lp - lm) / dd
        assert G[idx] == pytest.approx(fd, rel=2e-4, abs=1e-9)


def test_bf16_oracle_stays_close_to_fp64():
    params, norm, X, T = _data(B=16, seed=4)
    y64 = mlp.forward(params, norm, X, bf=False)
    y16 = mlp.forward(params, norm, X, bf=True)
    scale = np.abs(y64).max()
    assert np.abs(y16 - y64).max() < 3e-2 * scale
    _, g64 = mlp.grad(params, norm, X, T, bf=False)
    _, g16 = mlp.grad(params, norm, X, T, bf=True)
    cos = np.dot(g16, g64) / np.linalg.norm(g16) / np.linalg.norm(g64)
    assert cos > 0.995


def test_descriptor_hand_placed_cells():
    h = np.float32(0.01)
    R = np.float32(2) * h
    xg = np.array([0.5, 0.5, 0.5])
    pose_vel = np.arange(13, dtype=np.float32)
    # one fluid particle at the centre of cell (i, j, k) = (3, 0, 2), two in cell (0, 0, 0),
    # one boundary particle (ignored), one exactly on the lower face of cell (2, 2, 2)
    c320 = xg + (np.array([3, 0, 2]) - 2 + 0.5) * float(R)
    c000 = xg + (np.array([0, 0, 0]) - 2 + 0.25) * float(R)
    c000b = xg + (np.array([0, 0, 0]) - 2 + 0.75) * float(R)
    face = np.array([np.float32(np.float32(xg[0]) + np.float32(0) * R)] * 3, np.float32)
    x = np.array([c320, c000, c000b, c000, face], np.float32)
    v = np.array([[1, 2, 3], [1, 0, 0], [0, 2, 0], [9, 9, 9], [0, 0, 1]], np.float64)
    rho = np.array([1000.0, 900.0, 1100.0, 5.0, 950.0])
    m = np.array([1.0, 1.0, 3.0, 1.0, 2.0])
    fluid = np.array([1, 1, 1, 0, 1], np.int32)
    d = mlp.descriptor(x, v, rho, m, fluid, xg, pose_vel, h)
    np.testing.assert_array_equal(d[:13], pose_vel)
    cells = d[13:].reshape(64, 4)
    idx = lambda i, j, k: i + 4 * j + 16 * k
    np.testing.assert_allclose(cells[idx(3, 0, 2)], [1000, 1, 2, 3])
    np.testing.assert_allclose(cells[idx(0, 0, 0)], [1000, 0.25, 1.5, 0])      # mean rho; m-weighted v
    np.testing.assert_allclose(cells[idx(2, 2, 2)], [950, 0, 0, 1])            # lower face belongs
    occupied = {idx(3, 0, 2), idx(0, 0, 0), idx(2, 2, 2)}
    for c in range(64):
        if c not in occupied:
            assert np.all(cells[c] == 0)
