"""Error behaviour of the C ABI on the device path: calls out of order return
OSP_ESTATE, bad arguments OSP_EINVAL with the state unchanged, and every failure
leaves a message in osp_last_error."""
import ctypes as C

import numpy as np
import pytest

from paper_1712_00595_gb300 import native as N
from paper_1712_00595_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _status(fn, *args):
    return fn(*args)


def test_calls_out_of_order_and_bad_arguments():
    L = N.load_library()
    opt = N.osp_options()
    L.osp_default_options(C.byref(opt))
    opt.precision = 7  # no such precision
    h = C.c_void_p()
    assert L.osp_create(C.byref(h), C.byref(opt)) == N.OSP_EINVAL
    eng = N.Engine(precision=N.OSP_PREC_FP64, device=0)
    ops = np.zeros(1, W.UPDATE_DTYPE)
    out = np.zeros(4, np.float64)
    # nothing loaded yet
    assert L.osp_set_seeds(eng._h, N._ptr(np.array([0], np.int32)), 1, 0.15) == N.OSP_ESTATE
    assert L.osp_init_scores(eng._h, 1e-9, None) == N.OSP_ESTATE
    assert L.osp_apply_updates(eng._h, N._ptr(ops), 1, 1e-9, None) == N.OSP_ESTATE
    assert L.osp_query(eng._h, 0, 0, N._ptr(out)) == N.OSP_ESTATE
    assert L.osp_last_error(eng._h)
    # bad graphs
    src = np.array([0, 1, 2], np.int32)
    dst = np.array([1, 2, 5], np.int32)
    assert L.osp_load_graph(eng._h, 3, 3, N._ptr(src), N._ptr(dst), 0) == N.OSP_EINVAL
    assert L.osp_load_graph(eng._h, 0, 0, None, None, 0) == N.OSP_EINVAL
    src, dst = W.er_graph(50, 300, 4)
    eng.load_graph(50, src, dst)
    # seeds and c
    for seeds, c in (([0], 0.0), ([0], 1.0), ([50], 0.15), ([-2], 0.15), ([3, 3], 0.15)):
        a = np.array(seeds, np.int32)
        assert L.osp_set_seeds(eng._h, N._ptr(a), a.size, c) == N.OSP_EINVAL
    eng.set_seeds([0], 0.15)
    # no scores yet
    assert L.osp_apply_updates(eng._h, N._ptr(ops), 1, 1e-9, None) == N.OSP_ESTATE
    assert L.osp_topk(eng._h, 0, 5, 0, N._ptr(np.zeros(5, np.int32)), N._ptr(np.zeros(5)),
                      C.byref(C.c_int32())) == N.OSP_ESTATE
    assert L.osp_init_scores(eng._h, 0.0, None) == N.OSP_EINVAL
    eng.init_scores(1e-12)
    r0 = eng.query()
    # bad calls after init leave the scores as they were
    assert L.osp_apply_updates(eng._h, N._ptr(ops), 1, -1.0, None) == N.OSP_EINVAL
    assert L.osp_apply_updates(eng._h, N._ptr(ops), -1, 1e-9, None) == N.OSP_EINVAL
    assert L.osp_apply_updates(eng._h, None, 3, 1e-9, None) == N.OSP_EINVAL
    assert L.osp_query(eng._h, 1, 0, N._ptr(np.zeros(50))) == N.OSP_EINVAL
    assert L.osp_topk(eng._h, 0, 0, 0, N._ptr(np.zeros(1, np.int32)), N._ptr(np.zeros(1)),
                      C.byref(C.c_int32())) == N.OSP_EINVAL
    assert L.osp_topk(eng._h, 0, 4097, 0, N._ptr(np.zeros(4097, np.int32)),
                      N._ptr(np.zeros(4097)), C.byref(C.c_int32())) == N.OSP_EINVAL
    assert L.osp_export_graph(eng._h, 2, N._ptr(np.zeros(51, np.int64)),
                              N._ptr(np.zeros(300, np.int32))) == N.OSP_EINVAL
    assert L.osp_set_fixed_iterations(eng._h, -1) == N.OSP_EINVAL
    assert np.array_equal(eng.query(), r0)
    assert L.osp_last_error(eng._h)
    # an empty batch is a valid no-op
    st = eng.apply_updates(np.zeros(0, W.UPDATE_DTYPE), 1e-9)
    assert st["net_inserts"] == 0 and st["net_deletes"] == 0
    assert np.abs(eng.query() - r0).sum() <= 1e-14
    # status names
    assert L.osp_status_string(N.OSP_ETIMEOUT) == b"OSP_ETIMEOUT"
    eng.close()
    L.osp_destroy(None)  # accepted


def test_step_times_and_history_are_consistent():
    src, dst = W.er_graph(2000, 16000, 8)
    eng = N.Engine(precision=N.OSP_PREC_FP32_ACC64, device=0)
    eng.load_graph(2000, src, dst)
    eng.set_seeds([0], 0.15)
    st = eng.init_scores(1e-9)
    hist = eng.get_l1_history()
    times = eng.get_step_times()
    assert hist.size == st["iterations"] + 1 and times.size == st["iterations"] + 1
    assert hist[0] == pytest.approx(0.15, rel=1e-12)  # ||c e_s||_1
    assert hist[-1] <= 1e-9 < hist[-2]  # the do-while stop
    assert np.all(times > 0)
    eng.close()


def test_batch_stats_history_and_query_into_caller_buffer():
    rng = np.random.default_rng(12)
    src, dst = W.er_graph(3000, 24000, 9)
    eng = N.Engine(precision=N.OSP_PREC_FP32_ACC64, device=0, use_graphs=1)
    eng.load_graph(3000, src, dst)
    eng.set_seeds([0], 0.15)
    eng.init_scores(1e-9)
    es = W.EdgeSet(src, dst)
    dead = np.zeros(3000 + 64, np.uint8)
    for _ in range(3):
        ops, _ = W.random_mixed_batch(rng, 3000, es, dead, 40, p_add=0, p_delnode=0,
                                      protect=(0,))
        st = eng.apply_updates(ops, 1e-7)
        hist = eng.get_l1_history()
        # ||q_offset||_1 and ||x(k)||_1 of the call come from its step history
        assert hist.size == st["iterations"] + 1
        assert st["qoff_l1"] == hist[0] and st["last_x_l1"] == hist[-1]
        assert st["last_x_l1"] <= 1e-7
        # the scores written into a caller's (larger) buffer equal a fresh copy
        buf = np.full(5000, -1.0)
        got = eng.query(out=buf)
        assert got.size == 3000 and np.array_equal(got, eng.query())
        assert np.all(buf[3000:] == -1.0)
    with pytest.raises(ValueError):
        eng.query(out=np.zeros(10))
    with pytest.raises(ValueError):
        eng.query(out=np.zeros(5000, np.float32))
    eng.close()


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_waits_run_out_and_report_timeout(which):
    # failure detection without a GPU fault: a CTA that never reaches the grid
    # barrier (which 0) or a staged-row batch whose second row never lands
    # (which 1) ends in OSP_ETIMEOUT within the wait's limit, and the device
    # keeps working
    import time
    assert N.selftest_wait(which, False) == N.OSP_OK
    t0 = time.perf_counter()
    assert N.selftest_wait(which, True) == N.OSP_ETIMEOUT
    dt = time.perf_counter() - t0
    assert 1.0 < dt < 20.0
    src, dst = W.er_graph(500, 4000, 3)
    eng = N.Engine(precision=N.OSP_PREC_FP64, device=0)
    eng.load_graph(500, src, dst)
    eng.set_seeds([0, 1, 2], 0.15)
    eng.init_scores(1e-10)
    r = eng.query(0)
    assert np.all(np.isfinite(r)) and 0.5 < r.sum() <= 1 + 1e-9 and r[0] >= 0.15
    eng.close()
