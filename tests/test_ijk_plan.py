"""IJK-partitioned multi-process planning and exchange (Sec. III.A.1-III.A.3), on
CPU ranks: the library's host planner, the batched all-gather of step (v) over
gloo, and one distributed residual evaluation whose per-rank arithmetic is the
oracle's, checked against the single-process oracle."""
import os
import socket

import numpy as np
import pytest

from ._helpers import gpu_lib

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _lib():
    return gpu_lib()  # builds and loads librccsdt.so; the planner is host code


def _triples(o):
    out = []
    for k in range(o):
        for j in range(k + 1):
            for i in range(j + 1):
                out.append((i, j, k))
    return out


def _plan(o, v, ranks, batch, cost=None):
    from paper_2607_00981_gb300.distributed import IJKPlan
    return IJKPlan(_lib(), o, v, ranks, batch, cost)


@pytest.mark.parametrize("o,v,ranks,batch", [(1, 3, 1, 1), (3, 4, 2, 3), (4, 5, 3, 4), (6, 8, 4, 7),
                                             (16, 160, 8, 100), (16, 160, 5, 50)])
def test_plan_partitions_the_blocks(o, v, ranks, batch):
    p = _plan(o, v, ranks, batch)
    n3 = o * (o + 1) * (o + 2) // 6
    assert p.n3 == n3 and p.nbatches == min(n3, -(-n3 // batch))
    own = p.owners()
    assert own.min() >= 0 and own.max() < ranks
    # every block owned once; local lists are the owner map, in storage order
    seen = np.zeros(n3, dtype=int)
    for r in range(ranks):
        loc = p.local(r)
        assert (np.diff(loc) > 0).all() and (own[loc] == r).all()
        seen[loc] += 1
    assert (seen == 1).all()
    # the batches partition the blocks: each element is sent once per cycle
    sent = np.zeros(n3, dtype=int)
    for b in range(p.nbatches):
        counts, blocks = p.batch(b)
        assert counts.sum() == len(blocks) > 0
        owners = own[blocks]
        assert (np.diff(owners) >= 0).all()                       # grouped by owner, rank order
        assert (np.bincount(owners, minlength=ranks) == counts).all()
        for r in range(ranks):
            assert (np.diff(blocks[owners == r]) > 0).all()       # storage order inside a group
        sent[blocks] += 1
    assert (sent == 1).all()
    info_max_send = max(int(p.batch(b)[0].max()) for b in range(p.nbatches))
    assert p.max_send == info_max_send
    assert p.max_owned == max(len(p.local(r)) for r in range(ranks))
    p.close()


def test_default_cost_model_and_balance():
    lib = _lib()
    from paper_2607_00981_gb300.distributed import IJKPlan
    o, v = 16, 160
    c = IJKPlan.default_costs(lib, o, v)
    tr = _triples(o)
    full = 3 * v**5 + 15 * o * v**4 + 9 * v**4 + 3 * o * o * v**3 + 9 * o * v**3
    assert all(c[b] == (0.0 if i == k else full) for b, (i, j, k) in enumerate(tr))
    for ranks in (2, 3, 7, 8):
        p = IJKPlan(lib, o, v, ranks, 100)
        rc, bw = p.work()
        # longest-processing-time-first: loads differ by at most one block's cost
        assert rc.max() - rc.min() <= c.max()
        assert rc.sum() == pytest.approx(c.sum(), rel=1e-12)
        # per batch the step (v) work is spread over the ranks within a few percent
        assert (bw.max(1) / bw.mean(1)).max() < 1.10
        # and the batches carry equal shares of it
        tot = bw.sum(1)
        assert tot.max() / tot.mean() < 1.15
        p.close()


def test_step_v_work_counts_every_read_once():
    """Summed over batches, rank r's step (v) work is its computed blocks times the
    per-block reads: F_oo 3o and W_oooo 3o^2 reads of v^3 FMA, 15o ring reads of v^4."""
    lib = _lib()
    from paper_2607_00981_gb300.distributed import IJKPlan
    for o, v, ranks in ((3, 4, 2), (5, 7, 3), (9, 11, 4)):
        p = IJKPlan(lib, o, v, ranks, 5)
        own = p.owners()
        _, bw = p.work()
        per = (3 * o + 3 * o * o) * v**3 + 15 * o * v**4
        computed = np.array([i != k for (i, j, k) in _triples(o)])
        for r in range(ranks):
            assert bw[:, r].sum() == pytest.approx(per * np.sum(computed & (own == r)), rel=1e-12)
        p.close()


def test_user_costs_steer_the_ownership():
    lib = _lib()
    from paper_2607_00981_gb300.distributed import IJKPlan
    o = 6
    n3 = o * (o + 1) * (o + 2) // 6
    cost = np.ones(n3)
    cost[0] = n3 - 1.0          # one block as heavy as all the others together
    p = IJKPlan(lib, o, 4, 2, 8, cost)
    own = p.owners()
    assert (own == own[0]).sum() == 1     # its rank owns nothing else
    rc, _ = p.work()
    assert rc[0] == rc[1] == n3 - 1.0
    p.close()


def test_plan_rejects_bad_arguments():
    import ctypes as C
    lib = _lib()
    h = C.c_void_p()
    for args in ((0, 4, 2, 3), (65, 4, 2, 3), (4, 0, 2, 3), (4, 4, 0, 3), (4, 4, 4097, 3), (4, 4, 2, 0)):
        assert lib.rccsdt_ijk_plan_create(*args, None, C.byref(h)) == -1
    assert lib.rccsdt_ijk_plan_create(3, 4, 2, 3, None, None) == -1
    bad = np.ones(10)
    bad[3] = np.nan
    assert lib.rccsdt_ijk_plan_create(3, 4, 2, 3, bad.ctypes.data, C.byref(h)) == -1
    bad[3] = -1.0
    assert lib.rccsdt_ijk_plan_create(3, 4, 2, 3, bad.ctypes.data, C.byref(h)) == -1
    p = _plan(3, 4, 2, 3)
    n = C.c_int()
    assert lib.rccsdt_ijk_plan_local(p.h, 2, None, C.byref(n)) == -1
    counts = np.zeros(2, dtype=np.int32)
    assert lib.rccsdt_ijk_plan_batch(p.h, p.nbatches, counts.ctypes.data, None) == -1
    assert lib.rccsdt_ijk_block_costs(65, 4, np.zeros(1).ctypes.data) == -1
    p.close()


# ---------------------------------------------------------------------------
# gloo ranks
# ---------------------------------------------------------------------------

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _init(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _gather_worker(rank, world, port, o, v, batch, overlap, out):
    from paper_2607_00981_gb300 import synth
    from paper_2607_00981_gb300.distributed import IJKPlan, gather_batches
    _init(rank, world, port)
    try:
        import paper_2607_00981_gb300 as pkg
        plan = IJKPlan(pkg.load(build_if_missing=False), o, v, world, batch)
        t3c = synth.random_amplitudes_compact(o, v, seed=11)[2]
        loc = plan.local(rank)
        local = torch.from_numpy(t3c[loc].copy())
        got = torch.full((plan.n3, v, v, v), float("nan"), dtype=torch.float64)
        hits = np.zeros(plan.n3, dtype=int)
        order = []

        def consume(b, blocks, data):
            order.append(b)
            hits[blocks] += 1
            got[torch.as_tensor(blocks, dtype=torch.long)] = data

        sent = gather_batches(plan, rank, local, consume, overlap=overlap)
        out[rank] = (bool(torch.equal(got, torch.from_numpy(t3c))), hits.tolist(), order, sent, len(loc))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,o,v,batch,overlap", [(2, 4, 3, 3, True), (3, 5, 2, 4, True), (3, 4, 3, 2, False)])
def test_batched_allgather_delivers_every_block_once(world, o, v, batch, overlap):
    _lib()  # build before the ranks start
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_gather_worker, args=(world, port, o, v, batch, overlap, out), nprocs=world, join=True)
    n3 = o * (o + 1) * (o + 2) // 6
    for r in range(world):
        equal, hits, order, sent, nloc = out[r]
        assert equal                                  # bit-exact copy of the whole T3
        assert hits == [1] * n3                       # each block received once
        assert order == sorted(order) and sent == nloc
    assert sum(out[r][4] for r in range(world)) == n3


def _iteration_worker(rank, world, port, out):
    """Steps (iii)-(vii) of one distributed residual evaluation; the per-rank
    arithmetic is the oracle's (this process stands in for one rank's GPU)."""
    from oracle import compact as oc
    from oracle import rccsdt as full
    from paper_2607_00981_gb300 import synth
    from paper_2607_00981_gb300.distributed import IJKPlan, allreduce_sum_, gather_batches
    _init(rank, world, port)
    try:
        import paper_2607_00981_gb300 as pkg
        o, v, naux = 3, 4, 12
        inst = synth.make_instance(o, v, naux, seed=5)
        t1, t2, t3c = synth.random_amplitudes_compact(o, v, seed=6)
        plan = IJKPlan(pkg.load(build_if_missing=False), o, v, world, 3)
        loc = plan.local(rank)
        # (i)-(ii) replicated: dressing and the T2 parts of the intermediates
        Lt, ft = full.dress(inst.L, inst.fock_diag, t1)
        eri = full.Eri(Lt, o)
        I = full.intermediates(Lt, ft, t2, None, triples=True)
        # (iii) T3 parts of R1, R2 and W from the local blocks, summed over ranks
        mine = np.zeros_like(t3c)
        mine[loc] = t3c[loc]
        parts = [torch.from_numpy(np.ascontiguousarray(x)) for x in oc.t3_contributions(eri, ft, mine, o)]
        for x in parts:
            allreduce_sum_(x)
        dR1, dX2, dWvvvo, dWvooo = (x.numpy() for x in parts)
        I["Wvvvo"] = I["Wvvvo"] + dWvvvo
        I["Wvooo"] = I["Wvooo"] + dWvooo
        # (iv)-(v) the local residual blocks, the other ranks' T3 gathered in batches
        t3g = np.full_like(t3c, np.nan)

        def consume(b, blocks, data):
            t3g[blocks] = data.numpy()

        gather_batches(plan, rank, torch.from_numpy(t3c[loc].copy()), consume)
        r3loc = np.stack([oc.r3_block(I, t2, t3g, *oc.triples(o)[b]) for b in loc]) if len(loc) else \
            np.zeros((0, v, v, v))
        # (vi)-(vii) post-processing is block-local; the |R3|^2 shares are summed
        full_idx = np.zeros((o * (o + 1) * (o + 2) // 6, v, v, v))
        full_idx[loc] = r3loc
        r3p = oc.postprocess(full_idx, o)[loc]
        w = oc.weights(o)[loc]
        nrm = torch.tensor([float(np.sum(w * np.sum(r3p.reshape(len(loc), -1) ** 2, axis=1)))], dtype=torch.float64)
        allreduce_sum_(nrm)
        out[rank] = (loc.tolist(), r3loc, float(nrm[0]), dR1, dX2)
    finally:
        dist.destroy_process_group()


def test_distributed_residual_matches_the_single_process_oracle():
    from oracle import compact as oc
    from oracle import rccsdt as full
    from paper_2607_00981_gb300 import synth
    _lib()
    world = 3
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_iteration_worker, args=(world, port, out), nprocs=world, join=True)
    o, v, naux = 3, 4, 12
    inst = synth.make_instance(o, v, naux, seed=5)
    t1, t2, t3c = synth.random_amplitudes_compact(o, v, seed=6)
    r1, r2, r3c = oc.residuals_compact(inst.L, inst.fock_diag, t1, t2, t3c)
    Lt, ft = full.dress(inst.L, inst.fock_diag, t1)
    dR1, dX2, _, _ = oc.t3_contributions(full.Eri(Lt, o), ft, t3c, o)
    got = np.full_like(r3c, np.nan)
    for r in range(world):
        loc, r3loc, nrm, d1, d2 = out[r]
        got[loc] = r3loc
        np.testing.assert_allclose(d1, dR1, rtol=0, atol=1e-14)
        np.testing.assert_allclose(d2, dX2, rtol=0, atol=1e-14)
        r3n = oc.residual_norm(np.zeros_like(r1), np.zeros_like(r2), oc.postprocess(r3c, o), o)
        assert np.sqrt(nrm) == pytest.approx(r3n, rel=1e-13)
    np.testing.assert_allclose(got, r3c, rtol=0, atol=1e-13)
