"""Pins of the FP64 shower-shape oracle (Sec. 5.1 and App. A.1): a three-point
shower worked out by hand, points on an inclined axis, and the invariants
of a simulated batch."""
import math

import numpy as np

import oracle
from oracle import shapes
from paper_2202_05012_gb300 import inputs


def _res(x, y, z, E, offsets, layer_sum):
    return dict(x=np.array(x, float), y=np.array(y, float), z=np.array(z, float), E=np.array(E, float),
                offsets=np.array(offsets), layer_sum=np.array(layer_sum, float))


def test_three_points_by_hand():
    g = inputs.supa_d(2)  # slices 0-2: layer 0, 3-5: layer 1
    p = inputs.primaries(1, 0, e_lo=6.0, e_hi=6.0)
    p["x0"], p["y0"], p["theta"], p["phi"] = 0.0, 0.0, 0.0, 0.0
    res = _res([1, -1, 0], [0, 0, 2], [0, 1, 4], [3, 1, 2], [0, 3], [[4, 2]])
    lf, sf = shapes.shower_shapes(g, p, res)
    # layer 0: points (1, 0; E 3) and (-1, 0; E 1)
    np.testing.assert_allclose(lf[0, 0], [2, 4, 2 / 3, 0, 0, 1, 2, 1, 0, 0, 1, 0.5, 0, 1,
                                          math.sqrt(0.75), 0, 0, 0.5], atol=1e-15)
    # layer 1: one point (0, 2; E 2)
    np.testing.assert_allclose(lf[0, 1], [1, 2, 1 / 3, 0, 2, 2, 2, 0, 0, 0, 0, 0, 2, 2, 0, 0, 0, 1], atol=1e-15)
    np.testing.assert_allclose(sf[0], [6, 1, 2, 1 / 3, math.sqrt(2 / 9)], atol=1e-15)


def test_points_on_an_inclined_axis_have_no_lateral_extent():
    g = inputs.supa_d(3)
    p = inputs.primaries(1, 0, e_lo=5.0, e_hi=5.0)
    p["x0"], p["y0"], p["theta"], p["phi"] = 0.3, -0.2, 0.4, 1.1
    x0, y0, th, ph = (float(p[k][0]) for k in ("x0", "y0", "theta", "phi"))  # the float32 values
    t = math.tan(th)
    z = np.array([0.0, 2.0, 5.0, 7.0])
    res = _res(x0 + z * t * math.cos(ph), y0 + z * t * math.sin(ph), z, [1, 2, 1, 1], [0, 4], [[3, 1, 1]])
    lf, sf = shapes.shower_shapes(g, p, res)
    np.testing.assert_allclose(lf[0, :, 3:6], 0, atol=1e-12)
    np.testing.assert_allclose(lf[0, :, 11:14], 0, atol=1e-12)
    np.testing.assert_allclose(lf[0, :, 14:17], 0, atol=1e-6)  # sqrt of a rounding residue
    np.testing.assert_allclose(lf[0, :, 0], [2, 1, 1])
    np.testing.assert_allclose(sf[0, :4], [5, 2, 3, 0.6])


def test_invariants_of_a_simulated_batch():
    g = inputs.supa_d(30, grid=64, roi_mode=inputs.ROI_AXIS)
    p = inputs.primaries(100, 13, e_lo=1.0, e_hi=100.0, theta_max_deg=30.0, entry_halfwidth=0.25)
    res = oracle.simulate(g, p, 5, n_threads=8)
    lf, sf = shapes.shower_shapes(g, p, res)
    np.testing.assert_array_equal(lf[:, :, 0].sum(1), np.diff(res["offsets"]))
    np.testing.assert_allclose(lf[:, :, 1], res["layer_sum"], rtol=0, atol=0)
    np.testing.assert_allclose(lf[:, :, 2].sum(1), 1.0, rtol=1e-12)
    assert np.all(lf[:, :, 7:11] >= 0) and np.all(lf[:, :, 14:17] >= 0)
    assert np.all((lf[:, :, 17] >= 0) & (lf[:, :, 17] <= 1))
    occupied = lf[:, :, 0] > 0
    # the energy-weighted mean distance bounds the distance of the centroid
    assert np.all(np.hypot(lf[:, :, 11], lf[:, :, 12])[occupied] <= lf[:, :, 13][occupied] + 1e-12)
    assert np.all((sf[:, 3] >= 0) & (sf[:, 3] <= sf[:, 1]))
    np.testing.assert_allclose(sf[:, 0], res["layer_sum"].sum(1), rtol=1e-15)
