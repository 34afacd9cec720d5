"""The continuous-batching server: admission by slots and memory budget
(host logic, on the CPU with a stand-in solver), and on the GPU that each
request's result is the same alone and in the mix."""
import threading
import time

import numpy as np
import pytest

from paper_2110_13055_gb300 import cdi, inputs, serve


def _fake_solver(log, lock, fail_tag=None):
    state = {"running": 0, "max": 0}

    def solver(req):
        with lock:
            state["running"] += 1
            state["max"] = max(state["max"], state["running"])
        time.sleep(0.02 + 0.01 * (req.tag % 3))
        with lock:
            state["running"] -= 1
            log.append(req.tag)
        if req.tag == fail_tag:
            raise RuntimeError("bad request")
        return {"tag": req.tag}
    return solver, state


def test_admission_respects_slots_and_budget():
    log, lock = [], threading.Lock()
    solver, state = _fake_solver(log, lock, fail_tag=3)
    m = np.zeros((32, 64), np.uint8)
    need = serve.footprint_bytes(m, cdi.FP32)
    srv = serve.Server(slots=3, memory_budget=int(2.5 * need), solver=solver)
    reqs = [serve.Request(m, 1.0, 1e-4, 10, tag=i) for i in range(9)]
    for r in reqs:
        srv.submit(r)
    done = srv.drain(9, timeout=60)
    srv.close()
    assert len(done) == 9
    assert srv.max_running <= 2          # the memory budget holds two at a time
    assert srv.max_in_use <= 2.5 * need
    assert state["max"] <= 2
    failed = [r for r in done if r.error]
    assert [r.tag for r in failed] == [3]   # a bad request fails alone
    assert all(r.result["tag"] == r.tag for r in done if not r.error)


def test_oversized_request_is_rejected_not_blocking():
    log, lock = [], threading.Lock()
    solver, _ = _fake_solver(log, lock)
    big = np.zeros((256, 256), np.uint8)
    small = np.zeros((8, 8), np.uint8)
    srv = serve.Server(slots=2, memory_budget=serve.footprint_bytes(small, cdi.FP32) * 4,
                       solver=solver)
    srv.submit(serve.Request(big, 1.0, 1e-4, 1, tag=0))
    srv.submit(serve.Request(small, 1.0, 1e-4, 1, tag=1))
    done = srv.drain(2, timeout=30)
    srv.close()
    by = {r.tag: r for r in done}
    assert "budget" in by[0].error and not by[1].error


def test_footprint_grows_with_size_and_precision():
    a = np.zeros((32, 32), np.uint8)
    b = np.zeros((64, 64), np.uint8)
    assert serve.footprint_bytes(b, cdi.FP32) > serve.footprint_bytes(a, cdi.FP32)
    assert serve.footprint_bytes(a, cdi.FP32_SPLIT) > serve.footprint_bytes(a, cdi.FP32)
    assert serve.footprint_bytes(a, cdi.FP64) > serve.footprint_bytes(a, cdi.FP32_SPLIT)


@pytest.mark.gpu
def test_results_same_alone_and_in_the_mix():
    import __graft_entry__ as g
    g.build()
    masks = [inputs.grain_pack((32, 48), 0.6, 2.0, 4.0, seed=31)[0],
             inputs.grain_pack((12, 14, 16), 0.55, 1.5, 3.0, seed=32)[0],
             inputs.grain_pack((40, 40), 0.5, 2.0, 5.0, seed=33)[0],
             inputs.grain_pack((10, 12, 20), 0.5, 1.5, 3.0, seed=34)[0]]
    params = [(1.0, 1e-4), (1.2, 1e-6), (0.4, 3e-4), (0.8, 1e-5)]

    def make():
        return [serve.Request(m, V, U, 300, flow_tol=1e-7, max_flow_steps=20000, tag=i)
                for i, (m, (V, U)) in enumerate(zip(masks, params))]

    alone = [serve.solve(r) for r in make()]
    reqs = make()
    # a bad request in the mix (no pore cell in the inlet column) fails alone
    bad = masks[0].copy()
    bad[:, 0] = 1
    reqs.insert(2, serve.Request(bad, 1.0, 1e-4, 300, tag="bad"))
    done = serve.run_served(reqs, [0.0] * len(reqs), slots=4, memory_budget=8 << 30)
    by = {r.tag: r for r in done}
    assert "inlet" in by["bad"].error
    assert all(not r.error for r in done if r.tag != "bad")
    for r in done:
        if r.tag == "bad":
            continue
        a = alone[r.tag]
        assert np.array_equal(r.result["Gamma"], a["Gamma"])
        assert np.array_equal(r.result["C_out"], a["C_out"])


@pytest.mark.gpu
def test_served_result_matches_the_oracle():
    """One request served in a mix, in FP64 storage, against the oracle's
    run of the same request (flow, potential, transport, outputs)."""
    import __graft_entry__ as g
    import oracle as O
    g.build()
    m = inputs.grain_pack((24, 40), 0.6, 2.0, 4.0, seed=35)[0]
    other = inputs.grain_pack((10, 12, 16), 0.55, 1.5, 3.0, seed=36)[0]
    reqs = [serve.Request(m, 0.8, 1e-4, 400, precision=cdi.FP64, flow_tol=1e-8, tag=0),
            serve.Request(other, 1.2, 1e-6, 400, flow_tol=1e-7, max_flow_steps=20000, tag=1)]
    done = serve.run_served(reqs, [0.0, 0.0], slots=2, memory_budget=8 << 30)
    r = {q.tag: q for q in done}[0]
    assert not r.error
    o = O.run_case(m, flow_tol=1e-8, U_target=1e-4, applied_V=0.8, c0=10.0, psi_tol=1e-12,
                   n_np_steps=400)
    assert r.result["flow_steps"] == o["flow_steps"]
    np.testing.assert_allclose(r.result["Gamma"], o["Gamma"], rtol=1e-10)
    np.testing.assert_allclose(r.result["C_out"], o["C_out"], rtol=1e-10)


def test_first_fit_admission_and_ageing():
    """A small request that arrives behind a large one that does not fit yet
    starts first; a large request passed over max_bypass times is served
    next, before any younger small one."""
    log, lock = [], threading.Lock()
    small = np.zeros((64, 64), np.uint8)
    big = np.zeros((512, 512), np.uint8)
    ns, nb = serve.footprint_bytes(small, cdi.FP32), serve.footprint_bytes(big, cdi.FP32)
    assert nb > 2 * ns

    def solver(req):
        time.sleep(0.15 if req.tag == "big" else 0.05)
        with lock:
            log.append(req.tag)
        return {}

    srv = serve.Server(slots=2, memory_budget=nb, solver=solver, max_bypass=2)
    reqs = [serve.Request(small, 1.0, 1e-4, 1, tag="s0"),
            serve.Request(big, 1.0, 1e-4, 1, tag="big")]
    reqs += [serve.Request(small, 1.0, 1e-4, 1, tag=f"s{i}") for i in range(1, 6)]
    for r in reqs:
        srv.submit(r)
    done = srv.drain(len(reqs), timeout=60)
    srv.close()
    t = {r.tag: r.t_start for r in done}
    assert not any(r.error for r in done)
    assert t["s1"] < t["big"]                    # first fit: s1 did not wait for big
    passed = [k for k in ("s1", "s2", "s3", "s4", "s5") if t[k] < t["big"]]
    assert len(passed) <= 3                      # ageing: big is not passed over for ever
    assert max(t.values()) > t["big"]


def test_larger_requests_get_higher_stream_priority():
    """Stream priority grows one level per doubling of the footprint past
    256 MiB (lower numbers are served first); the server stamps it on each
    admitted request, or leaves 0 when prioritising is off."""
    mib = 1 << 20
    assert serve.size_priority(10 * mib) == 0
    assert serve.size_priority(300 * mib) == -1
    assert serve.size_priority(600 * mib) == -2
    assert serve.size_priority(1 << 40) == -5
    seen = {}

    def solver(req):
        seen[req.tag] = req.priority
        return {}
    small, big = np.zeros((32, 64), np.uint8), np.zeros((40, 160, 160), np.uint8)
    for flag in (True, False):
        seen.clear()
        srv = serve.Server(slots=2, memory_budget=64 << 30, solver=solver,
                           prioritise_large=flag)
        srv.submit(serve.Request(small, 1.0, 1e-4, 10, tag="small"))
        srv.submit(serve.Request(big, 1.0, 1e-6, 10, tag="big"))
        srv.drain(2, timeout=60)
        srv.close()
        want = serve.size_priority(serve.footprint_bytes(big, cdi.FP32)) if flag else 0
        assert seen == {"small": 0, "big": want}
        assert not flag or want < 0
