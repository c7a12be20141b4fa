"""Serving: requests of mixed kinds and sizes submitted together run concurrently on the server's
slots; every result equals the oracle's and equals the same request served alone (byte for byte);
a budget that admits one request at a time gives the same results; a request that can never fit
is refused at submission."""
import numpy as np
import pytest
import torch

import oracle
from helpers import sorted_ids
from paper_1704_00513_gb300 import build as fqbuild
from paper_1704_00513_gb300 import fqbfs
from paper_1704_00513_gb300 import inputs
from paper_1704_00513_gb300 import serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fqbuild.build()
    fqbfs.lib()


@pytest.fixture(scope="module")
def graphs():
    gs = []
    for scale, seed in ((13, 1), (15, 2)):
        off, cols = inputs.rmat_csr(scale, 16, seed=seed, device="cuda")
        gs.append((off, cols, inputs.pick_roots(off, 8, seed=seed)))
    return gs


def pinned_ids(ids_np):
    return torch.from_numpy(np.ascontiguousarray(ids_np.astype(np.uint32)).view(np.int32)).pin_memory()


def make_requests(graphs, gids):
    reqs, expect = [], []
    rng = np.random.default_rng(11)
    for i in range(36):
        kind = i % 3
        if kind == 0:
            g = i % len(graphs)
            off, cols, roots = graphs[g]
            root = roots[(i // 3) % len(roots)]
            r = serve.bfs_request(gids[g], root, off.numel() - 1, with_parent=True)
            expect.append(("bfs", g, root))
        elif kind == 1:
            ids = sorted_ids(int(rng.integers(1, 300_000)), float(rng.choice([1, 5, 80])), seed=i)
            r = serve.encode_request(pinned_ids(ids))
            expect.append(("enc", ids))
        else:
            ids = sorted_ids(int(rng.integers(0, 200_000)), float(rng.choice([2, 40])), seed=100 + i)
            st, stream = oracle.fq_encode(ids)
            r = serve.decode_request(torch.from_numpy(stream).pin_memory(), max(ids.size, 1))
            expect.append(("dec", ids))
        reqs.append(r)
    return reqs, expect


def result_bytes(r):
    # BFS parents are not unique (any valid tree is correct); they are validated separately
    if r.c.kind == serve.FQ_REQ_BFS:
        return r.depth.numpy().tobytes()
    if r.c.kind == serve.FQ_REQ_ENCODE:
        return r.out.numpy()[: r.c.out_count].tobytes()
    return r.out.numpy()[: r.c.out_count].tobytes()


def check_against_oracle(graphs, reqs, expect):
    host = [(o.cpu().numpy(), c.cpu().numpy().view(np.uint32)) for o, c, _ in graphs]
    for r, e in zip(reqs, expect):
        assert r.c.status == 0 and r.c.done == 1
        if e[0] == "bfs":
            off, cols = host[e[1]]
            ref, _ = oracle.bfs(off, cols, e[2])
            depth = r.depth.numpy()
            assert np.array_equal(depth, ref)
            assert oracle.validate(off, cols, e[2], depth, r.parent.numpy().view(np.uint32)) == 0
            assert r.c.out_count == (ref >= 0).sum()
        elif e[0] == "enc":
            st, ref = oracle.fq_encode(e[1])
            assert r.c.out_count == ref.size and np.array_equal(r.out.numpy()[: ref.size], ref)
        else:
            assert r.c.out_count == e[1].size
            assert np.array_equal(r.out.numpy()[: e[1].size].view(np.uint32), e[1])


def test_mixed_requests_concurrent_equal_alone_and_oracle(graphs):
    server = serve.Server(budget_bytes=16 << 30, slots=4, max_codec_ids=1 << 20)
    gids = [server.add_graph(o, c) for o, c, _ in graphs]
    reqs, expect = make_requests(graphs, gids)
    for r in reqs:
        server.submit(r)
    for r in reqs:
        st = server.wait(r)
        assert st == 0, (st, r.c.kind, hex(r.c.aux))
    # the requests overlapped: some started before others finished
    starts = sorted(r.c.t_start for r in reqs)
    ends = sorted(r.c.t_end for r in reqs)
    assert starts[len(starts) // 2] < ends[len(ends) // 2]
    check_against_oracle(graphs, reqs, expect)
    mixed = [result_bytes(r) for r in reqs]
    alone, _ = make_requests(graphs, gids)
    for r, m in zip(alone, mixed):
        server.submit(r)
        assert server.wait(r) == 0
        assert result_bytes(r) == m
    check_against_oracle(graphs, alone, expect)
    server.close()


def test_tight_budget_same_results(graphs):
    # room for the resident handles and one request's buffers only
    probe = serve.Server(budget_bytes=1 << 40, slots=3, max_codec_ids=1 << 20)
    [probe.add_graph(o, c) for o, c, _ in graphs]
    resident = probe.info()["resident"]
    probe.close()
    n_big = graphs[1][0].numel() - 1
    server = serve.Server(budget_bytes=resident + 8 * n_big + 4096 + (1 << 20) * 9, slots=3, max_codec_ids=1 << 20)
    gids = [server.add_graph(o, c) for o, c, _ in graphs]
    reqs, expect = make_requests(graphs, gids)
    for r in reqs:
        server.submit(r)
    for r in reqs:
        assert server.wait(r) == 0
    check_against_oracle(graphs, reqs, expect)
    huge = serve.encode_request(pinned_ids(np.arange(1 << 20, dtype=np.uint32)))
    huge.c.in_count = 1 << 36  # a footprint larger than the whole budget
    with pytest.raises(fqbfs.FqError) as e:
        server.submit(huge)
    assert e.value.status == fqbfs.FQ_ENOMEM
    server.close()
