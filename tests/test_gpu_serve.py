"""Request server (okmc_server_*): every result is the same alone and in the mix.

Each replica follows a script of solve and step requests.  Alone: the script runs on
its own handle, one call after another.  In the mix: all scripts are submitted at
once, interleaved, to a server with three lanes and a device budget that holds only
two of the replicas, so replicas are evicted and re-admitted between their requests.
Energies, positions and kinetic statistics must agree bit for bit (each replica's
computation is deterministic, and re-admission restores defects and kinetic state).
"""
import numpy as np
import pytest

import __graft_entry__
from paper_2403_09158_gb300 import okmc as ok
from paper_2403_09158_gb300.workload import scaled_population

pytestmark = pytest.mark.gpu

SMALL = dict(r111=(0.4, 1.0), r100=(0.4, 1.0))
KEYS = ('events', 'steps', 'negative_barriers', 'clock', 'dt_last')


@pytest.fixture(scope='module', autouse=True)
def _lib():
    __graft_entry__.build()
    ok.load()


def _replicas():
    specs = [((96, 96, 96), 60, 31, 450.0), ((64, 64, 64), 40, 32, 350.0), ((48, 48, 48), 25, 33, 550.0),
             ((32, 32, 32), 12, 34, 400.0), ((64, 64, 32), 20, 35, 500.0)]
    return [(scaled_population(n, nd, seed=s, **SMALL), T) for n, nd, s, T in specs]


SCRIPT = [('solve',), ('step', 4, ok.RESIDENCE), ('solve',), ('step', 3, ok.FIXED_DT), ('step', 2, ok.RESIDENCE),
          ('solve',)]


def _alone(w, T, seed):
    g = ok.Grid(w.n, w.voxel_nm, *w.C, seed=seed)
    g.set_defects(w.defects)
    out = []
    for req in SCRIPT:
        if req[0] == 'solve':
            out.append(('solve', g.interaction_energies(), g.stats()))
        else:
            st = g.step(T, req[1], mode=req[2])
            out.append(('step', g.get_positions(), st))
    g.close()
    return out


def test_results_same_alone_and_in_the_mix():
    reps = _replicas()
    alone = [_alone(w, T, 100 + i) for i, (w, T) in enumerate(reps)]
    est = [ok.estimate_field_bytes(w.n, w.voxel_nm, *w.C) for w, _ in reps]
    big = sorted(est)[-2:]
    budget = sum(big) + (6 << 20)  # the two largest replicas, with room for their defect tables
    assert budget < sum(est)
    srv = ok.Server(hbm_budget=budget, lanes=3)
    ids = [srv.add_replica(w.n, w.voxel_nm, *w.C, w.defects, seed=100 + i) for i, (w, T) in enumerate(reps)]
    tickets = [[] for _ in reps]
    for k, req in enumerate(SCRIPT):
        for i, (w, T) in enumerate(reps):
            if req[0] == 'solve':
                tickets[i].append(srv.submit_solve(ids[i]))
            else:
                tickets[i].append(srv.submit_step(ids[i], T, req[1], mode=req[2]))
    for i in range(len(reps)):
        for k, t in enumerate(tickets[i]):
            res, arr = srv.wait(t, timeout_ms=120000)
            assert res['status'] == ok.OKMC_OK, (i, k, res)
            kind, ref, st = alone[i][k]
            assert np.array_equal(arr, ref), (i, k, kind)
            for key in KEYS:
                assert res['stats'][key] == st[key], (i, k, key)
            assert res['t_submit'] <= res['t_start'] <= res['t_end']
    s = srv.stats()
    assert s['completed'] == s['submitted'] == len(reps) * len(SCRIPT)
    assert s['failed'] == 0
    assert s['evictions'] >= 1 and s['admissions'] > len(reps)
    assert s['device_bytes'] <= budget
    srv.close()


def test_server_rejects_bad_requests():
    w, T = _replicas()[3]
    srv = ok.Server(hbm_budget=0, lanes=1)
    rid = srv.add_replica(w.n, w.voxel_nm, *w.C, w.defects)
    with pytest.raises(ok.OkmcError):
        srv._submit(ok.Request(rid + 5, ok.SOLVE, 0, ok.StepParams(0.0, 0, 0, 0.0), None, None), None)
    with pytest.raises(ok.OkmcError):
        srv._submit(ok.Request(rid, 7, 0, ok.StepParams(0.0, 0, 0, 0.0), None, None), None)
    # a solve without an output array fails in the lane and reports it
    t = srv._submit(ok.Request(rid, ok.SOLVE, 0, ok.StepParams(0.0, 0, 0, 0.0), None, None), None)
    res, _ = srv.wait(t, timeout_ms=120000)
    assert res['status'] == ok.OKMC_EINVAL
    with pytest.raises(ok.OkmcError):
        srv.wait(t + 100, timeout_ms=0)
    # a replica larger than the budget is refused at registration
    small = ok.Server(hbm_budget=1 << 20, lanes=1)
    with pytest.raises(ok.OkmcError):
        small.add_replica(w.n, w.voxel_nm, *w.C, w.defects)
    small.close()
    srv.close()
