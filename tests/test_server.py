"""The serving engine (os3d_server_*): results equal direct calls, equal
whether a request runs alone or amid others, with graph replay or direct
launches, admission by arena footprint, bounded waits. Failures are made on
the host (a request that cannot fit, a wait that runs out), never on the GPU."""
import numpy as np
import pytest

from paper_1505_07690_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
MIX = [((32, 32, 32), 1), ((48, 48, 48), 0), ((64, 64, 64), 1), ((32, 48, 64), 0),
       ((32, 32, 32), 0), ((48, 48, 48), 1), ((16, 128, 160), 0)]


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_07690_gb300 import build, os3d
    build.build()
    return os3d


def _volumes():
    import torch
    return [torch.from_numpy(synth.straight_tubes(d, 3, seed=31 + i)).pin_memory()
            for i, (d, _) in enumerate(MIX)]


def _direct(M, vols):
    """The same transforms through os3d_forward / os3d_inverse on one stream."""
    import torch
    out = []
    for (d, sub), v in zip(MIX, vols):
        bank = M.os3d_make_wavelets(d, M.os3d_icosa_orientations(sub),
                                    M.os3d_default_params(L=12, overlap=0))
        fd = v.cuda().unsqueeze(0)
        out.append(M.os3d_inverse(bank, M.os3d_forward(bank, fd))[0].cpu().numpy())
    torch.cuda.synchronize()
    return out


def test_results_alone_and_in_the_mix_match_direct_calls(M):
    vols = _volumes()
    ref = _direct(M, vols)
    srv = M.Server(M.os3d_server_default_config(arena_bytes=2 << 30, max_inflight=3),
                   M.os3d_default_params(L=12))
    try:
        alone = []
        for (d, sub), v in zip(MIX, vols):           # one at a time
            t = srv.submit(v, sub)
            fo, lat = srv.wait(t, 60.0)
            assert lat > 0
            alone.append(fo.numpy().copy())
        tickets = [srv.submit(v, sub) for (d, sub), v in zip(MIX, vols)]   # all at once
        mixed = [srv.wait(t, 60.0)[0].numpy().copy() for t in tickets]
    finally:
        srv.close()
    for a, m, r in zip(alone, mixed, ref):
        assert rel(a, r) <= TOL
        assert rel(m, r) <= TOL
        assert rel(m, a) <= TOL


def test_admission_by_footprint_and_bounded_wait(M):
    import torch
    # room for one 64^3 x 42 request (score 88 MB + workspace) but not two
    srv = M.Server(M.os3d_server_default_config(arena_bytes=200 << 20, max_inflight=4),
                   M.os3d_default_params(L=12, block_slots=4))
    try:
        v = torch.from_numpy(synth.straight_tubes((64, 64, 64), 3, seed=5)).pin_memory()
        t1 = srv.submit(v, 1)
        t2 = srv.submit(v, 1)
        with pytest.raises(M.OS3DError) as e:
            srv.wait(t2, 0.0)          # queued behind t1: not done at once
        assert e.value.status == 4     # OS3D_ETIMEOUT, ticket still valid
        f1, _ = srv.wait(t1, 60.0)
        f2, _ = srv.wait(t2, 60.0)
        assert np.array_equal(f1.numpy(), f2.numpy())
        # a request whose footprint exceeds the whole arena completes with ENOMEM
        big = torch.zeros((128, 128, 128)).pin_memory()
        t3 = srv.submit(big, 2)
        with pytest.raises(M.OS3DError) as e:
            srv.wait(t3, 60.0)
        assert e.value.status == 2
    finally:
        srv.close()


def test_graph_replay_matches_direct_launches(M):
    """Repeated requests replay the captured graph of their (bank, home
    offset); results equal those of a server launching directly."""
    vols = _volumes()
    outs = {}
    for graphs in (1, 0):
        srv = M.Server(M.os3d_server_default_config(arena_bytes=2 << 30, max_inflight=1,
                                                    use_graphs=graphs),
                       M.os3d_default_params(L=12))
        try:
            res = []
            for _ in range(3):                       # the same sequence three times
                for (d, sub), v in zip(MIX, vols):
                    res.append(srv.wait(srv.submit(v, sub), 60.0)[0].numpy().copy())
            stats = srv.stats()
        finally:
            srv.close()
        outs[graphs] = res
        assert stats[0] == 3 * len(MIX)
        if graphs:
            # one stream slot and one request at a time: every request lands at
            # offset 0, the home of every bank; each bank is captured on its
            # first request and replayed by the second and third
            assert stats[1] == len(set(MIX))
            assert stats[2] == 2 * len(MIX)
        else:
            assert stats[1] == 0 and stats[2] == 0
    for a, b in zip(outs[1], outs[0]):
        assert np.array_equal(a, b)


def test_graph_replay_with_bf16_scores_and_streams(M):
    """BF16 score storage, three stream slots, requests in a mix: a replaying
    server returns what a directly launching one returns."""
    vols = _volumes()
    outs = {}
    for graphs in (1, 0):
        srv = M.Server(M.os3d_server_default_config(arena_bytes=2 << 30, max_inflight=3,
                                                    udtype=M.OS3D_U_BF16X2, use_graphs=graphs),
                       M.os3d_default_params(L=12))
        try:
            res = []
            for _ in range(3):
                tickets = [srv.submit(v, sub) for (d, sub), v in zip(MIX, vols)]
                res += [srv.wait(t, 60.0)[0].numpy().copy() for t in tickets]
            stats = srv.stats()
        finally:
            srv.close()
        outs[graphs] = res
        assert stats[0] == 3 * len(MIX)
    for a, b in zip(outs[1], outs[0]):
        assert np.array_equal(a, b)


def test_homes_give_replays_in_a_concurrent_mix(M):
    """Requests of a few banks arriving together: each bank's requests go back
    to the arena offsets its earlier requests used, so after the first round
    most requests replay a captured graph."""
    vols = _volumes()
    ref = _direct(M, vols)
    srv = M.Server(M.os3d_server_default_config(arena_bytes=2 << 30, max_inflight=3),
                   M.os3d_default_params(L=12))
    try:
        res = []
        for _ in range(6):
            tickets = [srv.submit(v, sub) for (d, sub), v in zip(MIX, vols)]
            res.append([srv.wait(t, 60.0)[0].numpy().copy() for t in tickets])
        done, captured, replayed = srv.stats()
    finally:
        srv.close()
    assert done == 6 * len(MIX)
    assert replayed >= 4 * len(MIX)
    for r in res:
        for a, b in zip(r, ref):
            assert rel(a, b) <= TOL


def test_bank_cache_budget_evicts_idle_banks(M):
    """With a bank budget smaller than any bank, every new bank evicts the idle
    ones; requests alternating between grids still return the direct results
    (evicted banks are rebuilt on their next use)."""
    vols = _volumes()
    ref = _direct(M, vols)
    srv = M.Server(M.os3d_server_default_config(arena_bytes=2 << 30, max_inflight=2,
                                                bank_cache_bytes=1),
                   M.os3d_default_params(L=12))
    try:
        for _ in range(2):
            tickets = [srv.submit(v, sub) for (d, sub), v in zip(MIX, vols)]
            out = [srv.wait(t, 60.0)[0].numpy().copy() for t in tickets]
            for a, b in zip(out, ref):
                assert rel(a, b) <= TOL
    finally:
        srv.close()
