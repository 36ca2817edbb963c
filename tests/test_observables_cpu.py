"""Host-side observables (no GPU): scalar order, periodic defect components, centroid."""
import numpy as np

from paper_2011_00287_gb300 import observables as OB


def _uniaxial(S, n, shape):
    Q = S * (np.outer(n, n) - np.eye(3) / 3)
    q5 = np.array([Q[0, 0], Q[0, 1], Q[0, 2], Q[1, 1], Q[1, 2]])
    return np.broadcast_to(q5.reshape(5, 1, 1, 1), (5,) + shape).copy()


def test_scalar_order_of_uniaxial_tensor():
    for S in (0.0, 0.3, 0.5):
        q5 = _uniaxial(S, np.array([0.6, 0.0, 0.8]), (2, 2, 2))
        np.testing.assert_allclose(OB.scalar_order(q5), S, atol=1e-14)


def test_defect_components_wrap_periodically():
    shape = (12, 12, 12)
    q5 = _uniaxial(0.5, np.array([1.0, 0, 0]), shape)
    psi = np.ones(shape)
    # a disordered blob split by the x seam counts once; a 2-site speck is ignored;
    # a disordered region outside the droplet (psi < 0) is ignored
    q5[:, 5:7, 5:7, 0:2] = 0.0
    q5[:, 5:7, 5:7, 11:12] = 0.0
    q5[:, 1, 1, 5:7] = 0.0
    q5[:, 9:11, 9:11, 8:10] = 0.0
    psi[9:11, 9:11, 8:10] = -0.8
    assert OB.defect_count(q5, psi) == 1
    # diagonal contact across a corner of the box joins two pieces (26-connectivity)
    q5b = _uniaxial(0.5, np.array([1.0, 0, 0]), shape)
    q5b[:, 0:2, 0:2, 0:2] = 0.0
    q5b[:, 10:12, 10:12, 10:12] = 0.0
    assert OB.defect_count(q5b, np.ones(shape)) == 1


def test_centroid_and_speed():
    L = (32, 32, 32)
    xs = np.array([[30.0, 1.0, 5.0], [31.0, 2.0, 5.0], [0.5, 3.0, 5.0], [1.5, 4.0, 5.0]])
    tr = OB.unwrap_trajectory(xs, L)
    np.testing.assert_allclose(tr[-1], [33.5, 4.0, 5.0])
    assert abs(OB.mean_speed(tr, 10.0) - np.mean([np.sqrt(2), np.sqrt(3.25), np.sqrt(2)]) / 10) < 1e-12
    # centroid from circular moments of a point mass at x = 3
    ang = 2 * np.pi * np.array([3.0, 7.0, 20.0]) / 32
    obs = np.zeros(12)
    obs[5:8], obs[8:11] = np.cos(ang), np.sin(ang)
    np.testing.assert_allclose(OB.centroid(obs, L), [3.0, 7.0, 20.0], atol=1e-12)
