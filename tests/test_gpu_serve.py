"""Serving: coalesced multi-handle queries and the request loop.

Integer work, so the tolerance is zero: every structure built inside the
serving mix must export the same bytes as the same build alone, and every query
answered in the mix (coalesced with others, while builds run) must equal the
same query answered alone."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_18497_b300 import build, phobic

    build.build()
    phobic.lib()
    return phobic


def _stream_keys(start, n, seed):
    from paper_2404_18497_b300 import workloads

    return workloads.stream_keys_torch(start, n, seed, "cuda")


def _negatives(n, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return torch.randint(-(2**62), 2**62, (n,), dtype=torch.int64, device="cuda", generator=g)


def test_query_multi_equals_separate_queries(ph):
    # phobic_query_multi decodes with the 64-bit partition arithmetic and
    # phobic_query, at these sizes, with the 32-bit one: this also checks the two
    # query instantiations against each other, for five encoders, both pilot
    # forms, members and non-members
    hs, keysets = [], []
    cfgs = [(7.0, 1.0, 2500, 0, 0), (7.0, 0.99, 2500, 1, 0), (6.0, 0.97, 1024, 1, 1), (8.0, 0.99, 4096, 0, 0),
            (7.0, 0.99, 2500, 2, 0), (7.0, 0.99, 2500, 7, 1), (7.0, 1.0, 2500, 6, 0)]
    for i, (lam, alpha, P, enc, mode) in enumerate(cfgs):
        k = _stream_keys(i * 10_000_000, 200_000 + 37_771 * i, 3)
        hs.append(ph.phobic_build_ex(k, ph.make_params(lam, alpha, P, encoder=enc, mode=mode)))
        keysets.append(k)
    rng = np.random.default_rng(4)
    reqs = []
    for r in range(40):
        i = int(rng.integers(0, len(hs)))
        m = int(rng.choice([0, 1, 7, 1000, 65_537, 300_001]))
        a = int(rng.integers(0, 3))  # unaligned starts too
        src = keysets[i] if r % 3 else _negatives(m + 3, r)  # members and non-members
        m = min(m, src.numel() - a)
        reqs.append((hs[i], src[a:a + m]))
    outs = [torch.full((k.numel() + 1,), -1, dtype=torch.int64, device="cuda")[1:] for _, k in reqs]
    ph.phobic_query_multi([h for h, _ in reqs], [k for _, k in reqs], outs)
    for (h, k), o in zip(reqs, outs):
        assert torch.equal(o, h.query(k))
    for h in hs:
        h.free()


def _alone(ph, keys, prm):
    h = ph.phobic_build_ex(keys, prm)
    return h, h.export()


def _run_mix(ph, srv, sets, prm, queries_per_set, seed):
    """Submits every build at once; as each completes, submits query batches
    against it (members and non-members) while other builds still run, then a
    release of every second MPHF.  Returns completions and the request records."""
    rng = np.random.default_rng(seed)
    torch.cuda.synchronize()
    bids = {srv.submit_build(k, prm): s for s, k in enumerate(sets)}
    built, qrec, done = {}, {}, []
    released = set()
    deadline = time.time() + 120
    while len(done) < len(bids) + len(qrec) + len(released) or len(built) < len(bids):
        assert time.time() < deadline, "serving mix did not finish"
        comp = srv.poll()
        if comp.size == 0:
            time.sleep(1e-4)
        for c in comp:
            done.append(c)
            if c["kind"] == ph.REQ_BUILD:
                assert c["status"] == ph.OK, c
                s = bids[int(c["request_id"])]
                built[s] = int(c["handle_id"])
                for q in range(queries_per_set):
                    m = int(rng.choice([1, 100, 4096, 50_000, 200_000]))
                    if q % 4 == 3:
                        keys = _negatives(m, 1000 * s + q)
                        torch.cuda.synchronize()
                    else:
                        a = int(rng.integers(0, max(1, sets[s].numel() - m)))
                        keys = sets[s][a:a + m]
                    out = torch.empty(keys.numel(), dtype=torch.int64, device="cuda")
                    qrec[srv.submit_query(built[s], keys, out)] = (s, keys, out)
            elif c["kind"] == ph.REQ_QUERY:
                s = qrec[int(c["request_id"])][0]
                # release every second MPHF once its own queries are all submitted
                if s % 2 == 1 and s not in released:
                    released.add(s)
                    srv.submit_release(built[s])
    srv.drain(60)
    done.extend(srv.poll())
    return bids, built, qrec, done, released


@pytest.mark.parametrize("serial", [False, True])
def test_server_results_same_alone_and_in_mix(ph, serial):
    sizes = [10_000, 3_000_000, 250_000, 1_200_000, 40_000, 2_000_000, 700_000, 15_000]
    sets = [_stream_keys(100_000_000 * (s + 1), n, 21) for s, n in enumerate(sizes)]
    prm = ph.make_params(7.0, 0.99, 2500, encoder=1)
    alone = [_alone(ph, k, prm) for k in sets]
    srv = ph.Server(build_slots=3, serial=serial)
    try:
        bids, built, qrec, done, released = _run_mix(ph, srv, sets, prm, 12, 5)
        # every MPHF that is still resident exports the same bytes as its build alone
        for s, hid in built.items():
            if s not in released:
                assert srv.handle(hid).export() == alone[s][1], s
        # every query answered in the mix equals the same query answered alone
        for rid, (s, keys, out) in qrec.items():
            assert torch.equal(out, alone[s][0].query(keys)), (s, rid)
        st = srv.stats()
        assert st["pending"] == 0 and st["queries_done"] == len(qrec) and st["builds_done"] == len(sets)
        assert st["resident_handles"] == len(sets) - len(released)
        arr = np.concatenate([np.atleast_1d(d) for d in done])
        qs = arr[arr["kind"] == ph.REQ_QUERY]
        assert (qs["status"] == ph.OK).all() and (qs["t_done_ns"] >= qs["t_submit_ns"]).all()
        if serial:
            assert (qs["batch_requests"] == 1).all()
        else:
            assert st["max_batch_requests_seen"] >= 1
        # a release completes after every query on its MPHF
        for s in released:
            rel = arr[(arr["kind"] == ph.REQ_RELEASE) & (arr["handle_id"] == built[s])]
            assert rel.size == 1
            mine = qs[qs["handle_id"] == built[s]]
            assert (mine["t_done_ns"] <= rel["t_done_ns"][0]).all()
    finally:
        srv.close()
        for h, _ in alone:
            h.free()


def test_server_coalesces_concurrent_queries(ph):
    """Many small batches against different MPHFs, submitted faster than one
    launch completes, share launches; each answer equals the answer alone."""
    sets = [_stream_keys(7_000_000_000 + s * 10_000_000, 100_000, 2) for s in range(6)]
    prm = ph.make_params(7.0, 1.0, 2500)
    srv = ph.Server(launch_slots=1)
    try:
        torch.cuda.synchronize()
        ids = [srv.submit_build(k, prm) for k in sets]
        srv.drain(60)
        hid = {int(c["request_id"]): int(c["handle_id"]) for c in srv.poll()}
        # one long batch first keeps the only launch slot busy while the rest queue up
        big = _negatives(250_000_000, 3)
        big_out = torch.empty_like(big)
        torch.cuda.synchronize()
        recs = [(0, big, big_out, srv.submit_query(hid[ids[0]], big, big_out))]
        for r in range(300):
            s = r % len(sets)
            k = sets[s][r * 97:r * 97 + 1 + r]
            o = torch.empty_like(k)
            recs.append((s, k, o, srv.submit_query(hid[ids[s]], k, o)))
        srv.drain(60)
        comp = srv.poll()
        assert (comp["status"] == ph.OK).all()
        assert comp["batch_requests"].max() > 1
        assert srv.stats()["query_launches"] < len(recs)
        for s, k, o, _ in recs:
            assert torch.equal(o, srv.handle(hid[ids[s]]).query(k))
    finally:
        srv.close()


def test_server_budget_admission(ph):
    """Under a budget that fits one build at a time, builds never overlap and
    the accounted bytes stay within the budget."""
    n = 2_000_000
    est = 32 * n + (64 << 20)
    budget = int(est * 1.5)
    sets = [_stream_keys(20_000_000_000 + s * 10_000_000, n, 8) for s in range(4)]
    prm = ph.make_params(7.0, 0.99, 2500, encoder=1)
    srv = ph.Server(hbm_budget_bytes=budget, build_slots=4)
    try:
        torch.cuda.synchronize()
        ids = {srv.submit_build(k, prm): i for i, k in enumerate(sets)}
        srv.drain(60)
        c = srv.poll()
        assert (c["status"] == ph.OK).all() and c.size == 4
        iv = sorted(zip(c["t_start_ns"].tolist(), c["t_done_ns"].tolist()))
        for (a0, a1), (b0, b1) in zip(iv, iv[1:]):
            assert a1 <= b0  # one at a time
        st = srv.stats()
        assert st["builds_waited_for_memory"] >= 1
        assert st["peak_accounted_bytes"] <= budget
        for rid, hid in zip(c["request_id"].tolist(), c["handle_id"].tolist()):
            alone = ph.phobic_build_ex(sets[ids[rid]], prm)
            assert srv.handle(hid).export() == alone.export()
            alone.free()
    finally:
        srv.close()


def test_server_ready_event_and_errors(ph):
    srv = ph.Server()
    try:
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            k = _stream_keys(30_000_000_000, 500_000, 4)
            ev = torch.cuda.Event()
            ev.record(s)
        rid = srv.submit_build(k, ph.make_params(7.0, 1.0, 2500), ready=ev)
        srv.drain(60)
        c = srv.poll()
        assert c.size == 1 and c["request_id"][0] == rid and c["status"][0] == ph.OK
        hid = int(c["handle_id"][0])
        with pytest.raises(ph.PhobicError) as e:
            srv.submit_query(hid + 1000, k, torch.empty_like(k))
        assert e.value.status == "INVALID_ARG"
        # a build with invalid parameters completes with that status
        srv.submit_build(k, ph.make_params(7.0, 1.5, 2500))
        srv.drain(60)
        c = srv.poll()
        assert c.size == 1 and c["status"][0] == 1 and c["handle_id"][0] == 0
        srv.submit_release(hid)
        with pytest.raises(ph.PhobicError):
            srv.submit_release(hid)  # already releasing
        with pytest.raises(ph.PhobicError):
            srv.submit_query(hid, k, torch.empty_like(k))
        srv.drain(60)
        assert srv.stats()["resident_handles"] == 0 and srv.stats()["resident_bytes"] == 0
    finally:
        srv.close()
