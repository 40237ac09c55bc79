"""Oracle self terms at full grid sizes, spread over a spawned process pool.

The sigma - W route of the oracle (energies_sampled) needs one real-space kernel per
unit eigenstrain tensor, which takes about a minute at 256^3; the kernels of the
tensors present are independent, so each worker builds one and evaluates the self
terms of the defects that share it.  Spawned processes (not forked) so that a pool
started after CUDA work in the parent is safe.  Test infrastructure: imports the
oracle only.
"""
import multiprocessing as mp
import os

import numpy as np

import oracle as O


def _group_tables(args):
    defects, n, h, C3, k0 = args
    C = O.stiffness_cubic(*C3)
    E, _ = O.unit_tensor(defects[0], h)
    K = O.unit_kernel(E, n, h, C, k0)
    return [O.self_term_table_realspace(d, n, h, K, O.unit_tensor(d, h)[1]) for d in defects]


def sampled_energies(defects, sample, sigma, n, h, C3, k0=O.MEAN_STRESS_ZERO):
    """{i: (e0, ec[8])} for the sampled defects, the oracle's sigma - W route with the
    total stress sigma (oracle layout) given."""
    groups = {}
    for i in sample:
        E, _ = O.unit_tensor(defects[i], h)
        groups.setdefault(tuple(np.round(E.ravel(), 12)), []).append(int(i))
    keys = list(groups)
    jobs = [([defects[i] for i in groups[k]], tuple(n), h, tuple(C3), k0) for k in keys]
    ctx = mp.get_context('spawn')
    with ctx.Pool(max(1, min(len(jobs), os.cpu_count() or 1))) as pool:
        tables = pool.map(_group_tables, jobs)
    out = {}
    for k, tabs in zip(keys, tables):
        for i, W in zip(groups[k], tabs):
            d = defects[i]
            c = O.pos_class(d['pos'])
            e0 = O.energy_of_stencil(d, d['pos'], sigma, h) - W[c, 0]
            ec = np.array([O.energy_of_stencil(d, Y, sigma, h) - W[c, 1 + j]
                           for j, Y in enumerate(O.candidate_positions(d['pos']))])
            out[i] = (e0, ec)
    return out
