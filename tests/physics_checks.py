"""Physical statements shared by the oracle pins and the GPU long-horizon tests (plain
numpy; no simulation code)."""
import numpy as np
from scipy.spatial.transform import Rotation


def three_balls(sc, z, fluid_z, fz, speed):
    """The buoyancy demo's ordering (Sec. 4: balls of density 0.1, 0.3 and 1.0 of the
    fluid's) after settling: lighter balls float higher, the two light ones with their
    centres above the free surface (a floating sphere of density ratio f has its centre
    R - d above it, d the cap depth holding f of its volume: 0.61 R for 0.1, 0.29 R for
    0.3), the neutral one below it; and each ball at rest with the fluid carrying its weight."""
    surface = np.percentile(fluid_z, 99)
    assert z[0] > z[1] + 0.008 and z[1] > z[2] + 0.02
    assert z[0] > surface + 0.015 and z[1] > surface + 0.005 and z[2] < surface
    weights = np.array([b.mass for b in sc.bodies[1:]]) * 9.81
    np.testing.assert_allclose(fz, weights, rtol=0.03)
    assert speed < 0.02


def top_momentum_energy(body_state, inertia_body):
    """World-frame angular momentum R I R^T w and rotational kinetic energy of a rigid body
    from its state row (t 3, q wxyz 4, v 3, w 3) and body-frame inertia."""
    st = np.asarray(body_state, np.float64)
    q = st[3:7]
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Iw, w = R @ np.asarray(inertia_body, np.float64) @ R.T, st[10:13]
    return Iw @ w, 0.5 * w @ Iw @ w


def asymmetric_top_scene():
    """A box spinning about no principal axis, no gravity, nothing else."""
    from paper_2511_15908_gb300 import scenes
    p = scenes.make_params(0.02, 1e-4, (-0.2, -0.2, -0.2), (0.2, 0.2, 0.2))
    p["g"] = (0.0, 0.0, 0.0)
    loc, _ = scenes.solid_box((0.04, 0.02, 0.06), 0.01)
    inertia = scenes._box_inertia(0.3, (0.04, 0.02, 0.06)).astype(np.float32)
    w0 = np.array([1.0, 0.5, 2.0], np.float32)
    b = scenes.Body(scenes.KIND_RIGID, loc, 0.01, mass=0.3, inertia=inertia,
                    pose=np.array([0, 0, 0, 1, 0, 0, 0], np.float32),
                    vel=np.array([0, 0, 0, *w0], np.float32))
    sc = scenes.Scene("top", p, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), 0.02, [b])
    return sc, inertia.astype(np.float64), w0.astype(np.float64)
