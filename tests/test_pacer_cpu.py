"""Publishing-rate control (host-side, no GPU): an offline source feeds a
two-stage chain -- a parallel stage of 3 servers (the GPU slots) followed by
one serial consumer that is the bottleneck (a fast but serial process, the
situation Section 3 of the paper describes) -- in a discrete-event
simulation driven by the native pacer.  Both policies keep the bottleneck
busy; the naive one (in-flight limit only) parks the whole in-flight budget
in front of the bottleneck, the smoothing one matches the publishing rate to
it with a fraction of the frames in flight and far lower latency."""
import heapq

import numpy as np
import pytest

N_FRAMES, SLOTS, LIMIT = 600, 3, 12
ALPHA, BETA = 1.0, 0.6          # parallel-stage and consumer time per unit of frame size


@pytest.fixture(scope="module")
def G():
    import paper_2502_09138_gb300.build as b
    b.build()
    import paper_2502_09138_gb300 as G
    return G


def simulate(G, policy):
    rng = np.random.default_rng(7)
    size = rng.uniform(0.5, 1.5, N_FRAMES)
    pacer = G.Pacer(policy, max_in_flight=LIMIT, initial_delay_s=0.05)
    ev = []                                   # (time, seq, kind, frame)
    seq = 0

    def push(t, kind, f=-1):
        nonlocal seq
        heapq.heappush(ev, (t, seq, kind, f))
        seq += 1

    now, nxt, consumed = 0.0, 0, 0
    q_a, q_b = [], []
    busy_a, busy_b = 0, False
    t_pub = np.zeros(N_FRAMES)
    t_done = np.zeros(N_FRAMES)
    busy_b_time = 0.0
    area_inflight, last_t = 0.0, 0.0
    retry_pending = False

    def in_flight():
        return nxt - consumed

    def backlog():
        # frames queued in front of the parallel stage, and beyond two waiting
        # at the consumer (enough to keep it busy across frame-size spread)
        return len(q_a) + max(0, len(q_b) - 2)

    def try_publish():
        nonlocal nxt, retry_pending, busy_a
        while nxt < N_FRAMES:
            ok, wait = pacer.try_publish(now, in_flight(), backlog())
            if not ok:
                if wait > 0 and not retry_pending:
                    push(now + wait, "retry")
                    retry_pending = True
                return
            t_pub[nxt] = now
            q_a.append(nxt)
            nxt += 1
            start_a()

    def start_a():
        nonlocal busy_a
        while busy_a < SLOTS and q_a:
            f = q_a.pop(0)
            busy_a += 1
            push(now + ALPHA * size[f], "done_a", f)

    def start_b():
        nonlocal busy_b
        if not busy_b and q_b:
            f = q_b.pop(0)
            busy_b = True
            push(now + BETA * size[f], "done_b", f)

    try_publish()
    while ev:
        t, _, kind, f = heapq.heappop(ev)
        area_inflight += in_flight() * (t - last_t)
        last_t = t
        now = t
        if kind == "retry":
            retry_pending = False
        elif kind == "done_a":
            busy_a -= 1
            q_b.append(f)
            start_a()
            start_b()
        elif kind == "done_b":
            busy_b = False
            busy_b_time += BETA * size[f]
            t_done[f] = now
            consumed += 1
            pacer.on_consumed(now, in_flight(), backlog())
            start_b()
        try_publish()
    lat = t_done - t_pub
    return dict(makespan=now, util_b=busy_b_time / now, inflight=area_inflight / now,
                p50=float(np.percentile(lat, 50)), p99=float(np.percentile(lat, 99)),
                delay=pacer.delay, pressure=pacer.pressure_events, mean_b=BETA * size.mean())


def test_smoothing_keeps_the_bottleneck_busy_with_fewer_frames_in_flight(G):
    naive = simulate(G, "naive")
    smooth = simulate(G, "smooth")
    # both run at the bottleneck's rate
    assert naive["util_b"] > 0.97, naive
    assert smooth["util_b"] > 0.95, smooth
    assert smooth["makespan"] < 1.08 * naive["makespan"], (smooth, naive)
    # naive parks the whole in-flight budget in the chain
    assert naive["inflight"] > 0.9 * LIMIT, naive
    assert smooth["inflight"] < 0.5 * naive["inflight"], (smooth, naive)
    assert smooth["p99"] < 0.65 * naive["p99"], (smooth, naive)
    # the adapted delay sits near the consumer's mean service time
    assert 0.65 * smooth["mean_b"] < smooth["delay"] < 1.6 * smooth["mean_b"], smooth


def test_naive_ignores_backlog_and_smooth_waits_for_its_delay(G):
    p = G.Pacer("naive", max_in_flight=2)
    assert p.try_publish(0.0, 0, 5)[0]            # backlog does not stop the naive source
    assert not p.try_publish(0.0, 2, 0)[0]        # the in-flight limit does
    s = G.Pacer("smooth", max_in_flight=4, initial_delay_s=1.0, decrease=0.1, increase=0.5)
    assert s.try_publish(10.0, 0, 0)[0]
    ok, wait = s.try_publish(10.25, 1, 0)
    assert not ok and abs(wait - 0.75) < 1e-12
    assert not s.try_publish(11.5, 1, 1)[0]       # back pressure
    s.on_consumed(12.0, 0, 0)
    assert abs(s.delay - 1.5) < 1e-12             # grew by (1 + increase)
    s.on_consumed(13.0, 0, 0)
    assert abs(s.delay - 1.35) < 1e-12            # shrank by (1 - decrease)
    assert s.pressure_events == 1


def test_invalid_configuration(G):
    with pytest.raises(Exception):
        G.Pacer("smooth", max_in_flight=0)
    with pytest.raises(Exception):
        G.Pacer("smooth", decrease=1.0)
