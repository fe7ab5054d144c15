"""Physical statements shared by the oracle pins and the GPU long-horizon tests (plain
numpy; no simulation code)."""
import numpy as np


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
