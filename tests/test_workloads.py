"""Host-side workload generators (CPU only): the learned closure's model
descriptors against values worked out by hand.

  * a homogeneous model has zero interface descriptors, and the damping
    descriptor is dt * sigma of the coarse sponge;
  * a flat interface between fine depths 2k and 2k + 1 (q1 above, q2 below,
    d = q2 - q1) is seen by coarse node k only: its full-weighting average is
    (3 q1 + q2) / 4, so the first descriptor is +d / 4, and the depth
    difference q(2k + 1) - q(2k - 1) is d; at coarse node k + 1 the fine
    nodes 2k + 1 .. 2k + 3 all hold q2;
  * an interface between fine depths 2k + 1 and 2k + 2 is seen by coarse
    node k + 1 only, with -d / 4 (its average (q1 + 3 q2) / 4 against its own
    q2) and depth difference d: the sign of the first descriptor tells on
    which side of the node the interface lies.
"""
import numpy as np
import pytest

from paper_1707_03776_gb300 import workloads as wl


def _fields(v_c, sigma=None):
    m_c = (1.0 / v_c ** 2).astype(np.float32)
    eta_c = np.zeros_like(m_c) if sigma is None else (m_c * sigma).astype(np.float32)
    return m_c, eta_c


def test_homogeneous_model_has_no_interface_descriptors():
    nc = 6
    v_c = np.full((nc,) * 3, 2000.0)
    v_f = np.full((2 * nc - 1,) * 3, 2000.0)
    sigma = wl.sponge_sigma((nc,) * 3, (20.0,) * 3, 2, 3500.0)
    m_c, eta_c = _fields(v_c, sigma)
    s = wl.closure_descriptors(v_c, v_f, eta_c, m_c, 1e-3, 3500.0)
    assert s.shape == (3, nc, nc, nc) and s.dtype == np.float32
    assert np.all(s[0] == 0.0) and np.all(s[1] == 0.0)
    np.testing.assert_allclose(s[2], 1e-3 * sigma, rtol=1e-6, atol=1e-9)
    assert s[2][nc // 2, nc // 2, nc // 2] == 0.0 and s[2].max() > 0


@pytest.mark.parametrize("last_fine_above,node,sign", [(6, 3, 1.0), (7, 4, -1.0)])
def test_flat_interface_is_seen_by_one_node(last_fine_above, node, sign):
    nc = 7
    v1, v2, vref = 1800.0, 3000.0, 3500.0
    zc = np.arange(nc)
    zf = np.arange(2 * nc - 1)
    v_c = np.broadcast_to(np.where(2 * zc <= last_fine_above, v1, v2), (nc, nc, nc)).astype(np.float64)
    v_f = np.broadcast_to(np.where(zf <= last_fine_above, v1, v2), (2 * nc - 1,) * 3).astype(np.float64)
    m_c, eta_c = _fields(v_c)
    s = wl.closure_descriptors(v_c, v_f, eta_c, m_c, 1e-3, vref)
    d = (v2 / vref) ** 2 - (v1 / vref) ** 2
    want0 = np.zeros(nc)
    want0[node] = sign * d / 4
    want1 = np.zeros(nc)
    want1[node] = d
    for i in (0, 3, nc - 1):
        for j in (0, 5):
            np.testing.assert_allclose(s[0][i, j], want0, rtol=1e-6, atol=1e-7)
            np.testing.assert_allclose(s[1][i, j], want1, rtol=1e-6, atol=1e-7)
    assert np.all(s[2] == 0.0)
