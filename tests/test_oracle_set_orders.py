"""Pins of the oracle's projection of the state to new orders (Sec. 2.4:
after each adaptation the solution is projected to the new polynomial
spaces): interpolation when the order rises, L2 projection when it falls."""
import numpy as np

from paper_2210_03523_gb300 import inputs as I
from oracle_helpers import tensor_weights


def test_raise_then_lower_is_identity(orc):
    mi = I.box_mesh(2, orders=I.random_orders(8, 1, 4, 41), phys=I.pulse_physics())
    m = orc.Mesh(mi)
    q = I.pulse_state(m.coords(), m.orders, mi.phys, width=0.4)
    hi = m.orders + np.array([2, 1, 3], dtype=np.int32)
    q_hi = m.set_orders(hi, q)
    m_hi = orc.Mesh(mi.with_orders(hi))
    back = m_hi.set_orders(m.orders, q_hi)
    np.testing.assert_allclose(back, q, rtol=0, atol=1e-13 * np.abs(q).max())


def test_lowering_keeps_element_integrals_and_low_degree_polynomials(orc):
    mi = I.box_mesh(2, geom_order=1, orders=(6, 5, 4), phys=I.pulse_physics())
    m = orc.Mesh(mi)
    q = I.pulse_state(m.coords(), m.orders, mi.phys, width=0.4)
    lo = np.tile(np.array([[3, 2, 4]], dtype=np.int32), (8, 1))
    ql = m.set_orders(lo, q)
    ml = orc.Mesh(mi.with_orders(lo))
    for e in range(8):
        a = (m.elem(q, e) * tensor_weights(m.orders[e])[None]).sum(1)
        b = (ml.elem(ql, e) * tensor_weights(lo[e])[None]).sum(1)
        np.testing.assert_allclose(b, a, rtol=1e-13)
    # a polynomial of degree <= the new orders survives unchanged
    poly = lambda x, y, z: np.stack([1 + x ** 3 + y * y * z, x, y, z, 2 + x * y * z])
    qp = I.pointwise_state(m.coords(), m.orders, poly)
    np.testing.assert_allclose(m.set_orders(lo, qp), I.pointwise_state(ml.coords(), lo, poly), atol=1e-13)
