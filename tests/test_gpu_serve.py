"""The continuous-batching server: every request's result equals the same
problem computed alone (indices bit-exact, values within the parity
tolerance), whatever batch it landed in; admission by memory splits the
stream into several batches; latency bookkeeping is consistent."""
import pytest
import torch

import oracle
import paper_2112_10223_gb300 as spk
import synth
from paper_2112_10223_gb300.serve import Request, Server, output_digest
from spk_testlib import compare, to_np

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    spk.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def pool():
    params = synth.batch_instance_params(12, seed=7, k_range=(2, 40), mn_range=(256, 4096), L_range=(4, 64))
    cpu = [synth.instance(p) for p in params]
    return cpu, [([tuple(t.to(DEV) for t in a) for a in A], m) for A, m in cpu]


@pytest.mark.parametrize("budget,batching", [(1 << 34, True), (3 << 20, True), (1 << 34, False)])
def test_served_results_match_the_oracle(pool, budget, batching):
    cpu, dev = pool
    seen = []

    def check(r):
        A, _ = cpu[r.tag]
        want = oracle.add(to_np(A))
        cp, ri, va = r.out
        compare((cp.cpu().numpy(), ri.cpu().numpy(), va.cpu().numpy()), want, va.dtype)
        seen.append((r.rid, r.batch_id))

    reqs = [Request(i, dev[i % len(dev)][0], dev[i % len(dev)][1], arrival=0.002 * i, tag=i % len(dev))
            for i in range(30)]
    st = Server(DEV, budget, batching=batching, on_done=check).run(reqs)
    assert sorted(r for r, _ in seen) == list(range(30))
    assert st.requests == 30 and len(st.latencies) == 30
    assert all(lat >= 0 for lat in st.latencies)
    if not batching:
        assert st.batches == 30
    if budget == 3 << 20:  # a few MB: batches must split
        assert st.batches > 1


def test_alone_vs_mix_digests_identical_indices(pool):
    _, dev = pool
    alone = [output_digest(spk.spkadd(A, m)) for A, m in dev]
    got = {}

    def keep(r):
        got[r.rid] = (r.tag, output_digest(r.out))

    reqs = [Request(i, dev[i % len(dev)][0], dev[i % len(dev)][1], arrival=0.0, tag=i % len(dev)) for i in range(24)]
    Server(DEV, 1 << 34, on_done=keep).run(reqs)
    for rid, (tag, d) in got.items():
        a = alone[tag]
        assert d[0] == a[0] and d[1] == a[1], rid
        assert abs(d[2] - a[2]) <= 1e-5 * max(a[3], 1.0)


def test_tight_budget_charges_exact_outputs(pool):
    """A budget of a few MB: batches are split, a request's output bound is replaced by its exact size after the
    symbolic phase, and the charge never passes the budget unless one request alone does."""
    cpu, dev = pool
    reqs = [Request(i, dev[i % len(dev)][0], dev[i % len(dev)][1], arrival=0.0, tag=i % len(dev))
            for i in range(24)]
    budget = 3 << 20
    srv = Server(DEV, budget)
    st = srv.run(reqs)
    one = max(r.bytes_bound() for r in reqs)
    assert st.batches > 1 and all(r.nnz_out >= 0 for r in reqs)
    assert srv.peak_charged <= max(budget, one)


def test_served_request_over_2pow31_output():
    """One served request whose B has more than 2^31 entries (int64 column pointers through the server)."""
    from spk_testlib import check_global_invariants, check_sampled, sample_columns

    m = n = 1 << 20
    A = synth.er(2, m, n, 1030, seed=21, dtype=torch.float32, device=torch.device(DEV))
    got = {}

    def keep(r):
        cp, ri, va = r.out
        check_global_invariants(A, (cp, ri, va), m)
        cols, _ = sample_columns(A, 32, 4, seed=3)
        last = torch.tensor([n - 2, n - 1], device=cp.device)
        check_sampled(A, (cp, ri, va), m, torch.unique(torch.cat([cols, last])), torch.float32)
        got["nnz"] = int(cp[-1].item())

    st = Server(DEV, 1 << 37, on_done=keep).run([Request(0, A, m, arrival=0.0)])
    assert st.requests == 1 and got["nnz"] > 2 ** 31
    del A
    torch.cuda.empty_cache()
