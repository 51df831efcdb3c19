"""Checkpoint and resume (dg_state_write / dg_state_info / dg_state_read):
host-only file I/O, so these run without a GPU.  A saved solution reads back
bit for bit with its orders and time; damaged, truncated, extended and
mismatched files are refused."""
import os

import numpy as np
import pytest

from paper_2210_03523_gb300 import inputs as I


@pytest.fixture(scope="module")
def dg():
    from paper_2210_03523_gb300 import build
    build.build()
    from paper_2210_03523_gb300 import dg as mod
    return mod


def _solution(seed=5):
    orders = I.random_orders(27, 1, 6, seed)
    n = int(sum((a + 1) * (b + 1) * (c + 1) for a, b, c in orders))
    q = np.random.default_rng(seed).standard_normal(5 * n)
    return orders, q


def test_round_trip_is_bitwise(dg, tmp_path):
    orders, q = _solution()
    p = tmp_path / "s.dgs"
    dg.save_state(p, orders, q, t=0.123456789)
    o2, q2, t2 = dg.load_state(p)
    assert np.array_equal(o2, orders)
    assert q2.tobytes() == q.tobytes()
    assert t2 == 0.123456789
    assert os.path.getsize(p) == 8 + 4 + 4 + 8 + 8 + 4 * orders.size + 8 * q.size + 8


def test_special_values_survive(dg, tmp_path):
    orders = np.array([[1, 1, 1]], dtype=np.int32)
    q = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, 1.7976931348623157e308, 1.0] * 5)
    p = tmp_path / "v.dgs"
    dg.save_state(p, orders, q, t=-2.5)
    _, q2, t2 = dg.load_state(p)
    assert q2.tobytes() == q.tobytes() and t2 == -2.5


def test_damaged_files_are_refused(dg, tmp_path):
    orders, q = _solution(6)
    p = tmp_path / "s.dgs"
    dg.save_state(p, orders, q, t=1.0)
    raw = p.read_bytes()
    cases = {
        "bit flip in the state": raw[:200] + bytes([raw[200] ^ 1]) + raw[201:],
        "bit flip in an order": raw[:33] + bytes([raw[33] ^ 4]) + raw[34:],
        "bit flip in the time": raw[:24] + bytes([raw[24] ^ 1]) + raw[25:],
        "truncated": raw[:-9],
        "trailing bytes": raw + b"\0",
        "wrong magic": b"XGSTATE1" + raw[8:],
        "wrong version": raw[:8] + (2).to_bytes(4, "little") + raw[12:],
        "empty": b"",
    }
    for why, data in cases.items():
        bad = tmp_path / "bad.dgs"
        bad.write_bytes(data)
        with pytest.raises(dg.DGError):
            dg.load_state(bad)
            pytest.fail(why)


def test_argument_checks(dg, tmp_path):
    import ctypes as C
    lib = dg._lib()
    orders, q = _solution(7)
    p = str(tmp_path / "s.dgs").encode()
    o = np.ascontiguousarray(orders, dtype=np.int32)
    op = o.ctypes.data_as(C.POINTER(C.c_int32))
    qp = q.ctypes.data_as(C.POINTER(C.c_double))
    assert lib.dg_state_write(None, o.shape[0], op, qp, 0.0) == 1
    assert lib.dg_state_write(p, 0, op, qp, 0.0) == 1
    assert lib.dg_state_write(p, o.shape[0], None, qp, 0.0) == 1
    bad = o.copy()
    bad[0, 0] = 0
    assert lib.dg_state_write(p, o.shape[0], bad.ctypes.data_as(C.POINTER(C.c_int32)), qp, 0.0) == 1
    assert lib.dg_state_write(str(tmp_path / "no" / "dir.dgs").encode(), o.shape[0], op, qp, 0.0) == 1
    assert lib.dg_state_write(p, o.shape[0], op, qp, 0.0) == 0
    # a reader that expects another element count
    o2 = np.empty((o.shape[0] + 1, 3), dtype=np.int32)
    q2 = np.empty(q.size + 1000)
    assert lib.dg_state_read(p, o.shape[0] + 1, o2.ctypes.data_as(C.POINTER(C.c_int32)),
                             q2.ctypes.data_as(C.POINTER(C.c_double)), None) == 1
    assert lib.dg_state_read(str(tmp_path / "missing.dgs").encode(), o.shape[0], op, qp, None) == 1
    assert lib.dg_state_info(None, None, None, None) == 1
    assert lib.dg_state_info(p, None, None, None) == 0
