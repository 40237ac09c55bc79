"""Benchmark: OkMC residence-time steps with exact FFT elastic interactions.

One step = one pass of the whole hot path on the 256^3 workload (2000 defects):
incremental eigenstrain update of the moved defect, forward R2C transform of the
six eigenstrain components, Green operator, inverse C2R transform, interaction
energies at every defect site and after each of the eight jumps, rates, one
residence-time event.  Metric: voxel stress+energy updates per second
(N voxels x steps / s); OkMC events/s and the HBM roofline fraction of the
dominant kernel are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica (replicas only: the path has
no exchange step); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = 'voxel stress+energy updates/s'
UNIT = 'voxel updates/s'


def _peaks():
    p = os.path.join(ROOT, 'MEASURED_PEAKS.json')
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d['hbm_gbs']), 'measured'
    return 6800.0, 'fallback'


def max_over_ranks(x, ws):
    """The largest value of x over the ranks (the job takes as long as its slowest
    replica); x itself when there is one rank."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    if ws > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _dist():
    ws = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    return ws, rank


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile('w+', suffix='.csv', delete=False)
        q = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,'
             'clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,'
             'clocks_event_reasons.sw_power_cap')
        try:
            self.p = subprocess.Popen(['nvidia-smi', '-i', str(gpu_index), '--query-gpu=' + q, '--format=csv,noheader,nounits',
                                       '-lms', '100'], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['nvidia-smi unavailable']}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(',') for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace('.', '').isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace('.', '').isdigit()]
        reasons = set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        for r in rows:
            if len(r) < 9:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == 'active':
                    reasons.add(nm)
        return {'sm_mhz': statistics.median(sm) if sm else None, 'sm_max_mhz': max(mx) if mx else None,
                'reasons': sorted(reasons), 'samples': len(sm)}


def kernel_bytes(name, n):
    """Algorithmic HBM bytes of one launch (FP32 fields, int32 fixed-point eigenstrain):
    each pass reads and writes the six-component field once."""
    nx, ny, nz = n
    N = nx * ny * nz
    spec = 6 * nz * (nx // 2 + 1) * ny * 8
    return {'plane_fwd': 6 * N * 4 + spec, 'pencil_green': 2 * spec, 'plane_inv': spec + 6 * N * 4}.get(name)


def cufft_reference(n, stream, reps):
    """Device time (ms) of cuFFT (through torch.fft) on the same transform sizes: a
    forward R2C and an inverse C2R of six components of an n grid, without the Green
    operator.  A reference point for the solve passes; the library does not use it."""
    import torch
    x = torch.randn((6, n[2], n[1], n[0]), device='cuda', dtype=torch.float32)
    for _ in range(2):
        y = torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)), s=(n[2], n[1], n[0]), dim=(1, 2, 3))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        y = torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)), s=(n[2], n[1], n[0]), dim=(1, 2, 3))
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del x, y
    torch.cuda.empty_cache()
    return ms


def run_ours(args, ws, rank):
    import ctypes as C

    import torch

    from paper_2403_09158_gb300 import okmc as ok
    from paper_2403_09158_gb300.workload import config_large

    torch.cuda.set_device(int(os.environ.get('LOCAL_RANK', '0')))
    dev = torch.cuda.current_device()
    w = config_large(seed=1003 + rank)
    stream = torch.cuda.current_stream()
    g = ok.Grid(w.n, w.voxel_nm, *w.C, precision=ok.FP32_FIELDS, seed=20231 + rank, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    g.set_defects(w.defects)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    N = int(np.prod(w.n))
    for _ in range(args.warmup):
        g.step(w.T_K, 1)
    torch.cuda.synchronize()
    stats0 = g.stats()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # timed region: each step is one replay of the captured step graph.  The region of
    # exactly K steps gives `value`; the same K-step region is then repeated until about a
    # second has passed, inside the same clock record, so that the clocks are sampled
    # under load and the spread of the K-step time is known.
    clk = Clocks(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        g.step(w.T_K, 1)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    stats1 = g.stats()
    events = stats1['events'] - stats0['events']
    repeats = []
    t_rep = time.perf_counter()
    while time.perf_counter() - t_rep < 1.0 and len(repeats) < 1000:
        ev0.record(stream)
        for _ in range(args.steps):
            g.step(w.T_K, 1)
        ev1.record(stream)
        torch.cuda.synchronize()
        repeats.append(ev0.elapsed_time(ev1))
    clocks = clk.stop()
    # second timed region of the same length: kernel by kernel, each launch between
    # CUDA events on the handle's stream (per-kernel durations for the roofline)
    g.reset_kernel_times()
    g.set_profiling(True)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        g.step(w.T_K, 1)
    torch.cuda.synchronize()
    g.set_profiling(False)
    kt = g.kernel_times()
    # end to end through the C ABI with host buffers: the step's input positions in
    # from pinned host memory, one step, the moved positions and the step statistics
    # (clock, events) out
    pos_h = torch.from_numpy(g.get_positions()).pin_memory()
    pos_out = torch.empty_like(pos_h).pin_memory()
    torch.cuda.synchronize()
    k_e2e = max(3, args.steps // 2)
    lat = []
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        t1 = time.perf_counter()
        g.set_positions(pos_h.numpy())
        g.step(w.T_K, 1)                 # returns the step statistics (clock, events) read back
        g.get_positions(pos_out.numpy())
        pos_h.copy_(pos_out)
        lat.append(time.perf_counter() - t1)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / k_e2e
    # request latency over a longer run of the same end-to-end step (host clock)
    for _ in range(max(0, 200 - k_e2e)):
        t1 = time.perf_counter()
        g.set_positions(pos_h.numpy())
        g.step(w.T_K, 1)
        g.get_positions(pos_out.numpy())
        pos_h.copy_(pos_out)
        lat.append(time.perf_counter() - t1)
    # a full solve: every plane transformed (as after okmc_set_defects, or a fixed-time
    # step that moves many defects), timed kernel by kernel on the handle's stream
    full = []
    for _ in range(3):
        g.set_defects(w.defects)
        torch.cuda.synchronize()
        g.reset_kernel_times()
        g.set_profiling(True)
        g.solve_stress(copy=False)
        torch.cuda.synchronize()
        g.set_profiling(False)
        kf = g.kernel_times()
        full.append({k: kf[k][0] / kf[k][1] for k in ('plane_fwd', 'pencil_green', 'plane_inv') if k in kf})
    g.close()
    cufft = cufft_reference(w.n, stream, max(3, args.steps // 3))
    ms = max_over_ranks(ms, ws)
    e2e_s = max_over_ranks(e2e_s, ws)
    return dict(ms=ms, N=N, events=events, kt=kt, clocks=clocks, setup_s=setup_s, e2e_s=e2e_s, cufft=cufft,
                nd=len(w.defects), n=w.n, T=w.T_K, stats_bytes=C.sizeof(ok.StepStats), repeats=repeats,
                lat_ms=[x * 1e3 for x in lat], full=full)


def _time_steps(g, T, steps, stream):
    """Device time (ms) of `steps` residence steps (graph replays) and the events they ran."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ev = g.stats()['events']
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        g.step(T, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), g.stats()['events'] - ev


def run_dipole(args):
    """Exact against dipole-approximation interaction energy of two 1/2<111> loops (the
    loop-loop geometry of the paper's Sec. 4: radius 3.3 nm, Burgers vectors and normals
    along [111]; one loop fixed at the centre of a 128^3 box, the other 10 nm away along
    [1-10] and moved along its glide direction [111]).  For each position: the exact
    energy (Eq. interaction_energy3) and the dipole one (Eq. interaction_energy4) of the
    moving loop, and the time of one evaluation after the move (the incremental solve,
    both energies and their copies to the host).  Then the paper's shift-theorem
    evaluation of the same loop at 121 continuous positions along the glide line."""
    import torch

    from paper_2403_09158_gb300 import okmc as ok
    from paper_2403_09158_gb300.workload import LOOP_111, ONE_D, make_defects

    n = (128, 128, 128)
    h = 0.2855
    c0 = np.array([128, 128, 128])
    off = np.array([50, -50, 0])                      # 10.09 nm along [1-10]
    steps = list(range(-60, 61, 6))                   # half-lattice steps along [111]
    defs = make_defects([LOOP_111, LOOP_111], np.array([c0, c0 + off + steps[0]]), [0, 0], [3.3, 3.3], [0, 0],
                        [0.1, 0.1], [ONE_D, ONE_D])
    stream = torch.cuda.current_stream()
    clk = Clocks(torch.cuda.current_device())
    rows = []
    g = ok.Grid(n, h, 243.0, 145.0, 116.0, precision=ok.FP32_FIELDS, stream=stream.cuda_stream)
    g.set_defects(defs)
    pos = g.get_positions()
    E = np.zeros(2)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    g.interaction_energies(E)                         # warm-up
    for k in steps:
        pos[1] = (c0 + off + k) % (2 * np.asarray(n))
        g.set_positions(pos)                          # the moved loop's planes become dirty
        torch.cuda.synchronize()
        e0.record(stream)
        g.solve_stress(copy=False)                    # incremental: the dirty planes only
        Ex = g.interaction_energies()
        Ed, _ = g.dipole_energies()
        e1.record(stream)
        torch.cuda.synchronize()
        rows.append((k * math.sqrt(3.0) * h / 2.0, float(Ex[1]), float(Ed[1]), e0.elapsed_time(e1)))
    xs = [r[0] for r in rows]
    # the paper's own evaluation (Sec. 3.3, Eq. shift): the moving loop's field translated
    # to continuous positions along its glide line; on the lattice sites above it gives
    # the stencil energies back (up to the Nyquist terms of the even edges)
    u = np.ones(3) / math.sqrt(3.0)
    centre = (c0 + off) * h / 2.0
    xc = np.linspace(xs[0], xs[-1], 121)
    torch.cuda.synchronize()
    e0.record(stream)
    Es = g.shift_energies(1, centre[None, :] + xc[:, None] * u[None, :])
    e1.record(stream)
    torch.cuda.synchronize()
    ms_shift = e0.elapsed_time(e1)
    Es_sites = g.shift_energies(1, centre[None, :] + np.asarray(xs)[:, None] * u[None, :])
    g.close()
    gap = max(abs(r[1] - r[2]) for r in rows)
    far = [abs(r[1] - r[2]) / max(1e-12, abs(r[1])) for r in rows if abs(r[0]) > 12.0]
    out = {'metric': 'exact vs dipole interaction energy, two 1/2<111> loops', 'unit': 'eV',
           'data': 'synthetic', 'dtype': 'f32 fields / f64 energies',
           'config': {'workload': 'loop_loop_128cubed (R = 3.3 nm loops, b || n || [111], 10.09 nm apart along '
                                  '[1-10], the second moved along [111]; Fe cubic C11/C12/C44 = 243/145/116 GPa)'},
           'x_nm': xs, 'E_exact_eV': [r[1] for r in rows], 'E_dipole_eV': [r[2] for r in rows],
           'max_abs_gap_eV': gap, 'rel_gap_beyond_12nm_max': max(far) if far else None,
           'ms_per_evaluation_median': float(np.median([r[3] for r in rows])),
           'shift_x_nm': xc.tolist(), 'E_shift_eV': Es.tolist(),
           'shift_minus_exact_at_sites_max_abs_eV': float(np.abs(Es_sites - np.array([r[1] for r in rows])).max()),
           'ms_shift_call_121_positions': ms_shift,
           'evaluation': 'after each move: incremental solve, exact and dipole energies, both copied to the host',
           'clocks': clk.stop()}
    print(json.dumps(out))
    return 0


def _loop_ensemble(ok, w, runs, steps, every, stream, lines=None):
    """`runs` seeded replicas of workload w (optionally in the field of immobile
    dislocation lines) advanced as one batch by `steps` fixed-time-step steps (Algorithm
    1); every `every` steps the loops' coordinates along [111] (unwrapped, nm) and the
    clock.  Returns (trajectories (runs, K, n_defects), clock (runs, K), seconds)."""
    import torch

    unit = 0.5 * w.voxel_nm
    grids = []
    for r in range(runs):
        g = ok.Grid(w.n, w.voxel_nm, *w.C, seed=2000 + r, stream=stream.cuda_stream)
        if lines:
            g.set_dislocations(lines)
        g.set_defects(w.defects)
        grids.append(g)
    batch = ok.Batch(grids, stream=stream.cuda_stream)
    p0 = grids[0].get_positions().astype(np.int64)
    tr = np.zeros((runs, steps // every + 1, len(w.defects)))
    clock = np.zeros((runs, steps // every + 1))
    tr[:, 0] = (p0 @ np.ones(3)) * unit / math.sqrt(3.0)
    box = 2 * np.asarray(w.n)
    t0 = time.perf_counter()
    for k in range(1, steps // every + 1):
        st = batch.step(w.T_K, every, mode=ok.FIXED_DT)
        for r, g in enumerate(grids):
            d = g.get_positions().astype(np.int64) - p0
            d -= np.round(d / box).astype(np.int64) * box          # unwrap the periodic moves
            tr[r, k] = ((p0 + d) @ np.ones(3)) * unit / math.sqrt(3.0)
            clock[r, k] = st[r]['clock']
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    batch.close()
    for g in grids:
        g.close()
    return tr, clock, seconds


def _trajectory_summary(tr, clock):
    out = {'time_ns': (clock.mean(axis=0) * 1e9).tolist()}
    for i in range(tr.shape[2]):
        out['x%d_mean_nm' % (i + 1)] = tr[:, :, i].mean(axis=0).tolist()
        out['x%d_envelope_nm' % (i + 1)] = [tr[:, :, i].min(axis=0).tolist(), tr[:, :, i].max(axis=0).tolist()]
    return out


def run_kinetics(args):
    """The paper's two-loop kinetics (Sec. 5.1): two 1/2<111> loops 10 nm apart across
    their glide axis and x_rel = 10 nm (inside the attraction well) or 20 nm (outside it)
    along it; 500 fixed-time-step steps (Algorithm 1, dt from the nominal barrier) at
    300 K, 10 runs per case as one batch of replicas with different seeds.  Reports the
    mean and the envelope of both loops' coordinates along [111] against time."""
    import torch

    from paper_2403_09158_gb300 import okmc as ok
    from paper_2403_09158_gb300.workload import config_kinetics

    runs, steps, every = 10, 500, 10
    stream = torch.cuda.current_stream()
    clk = Clocks(torch.cuda.current_device())
    cases = []
    t_total = 0.0
    for x_rel in (10.0, 20.0):
        w = config_kinetics(x_rel, n=args.box)
        tr, clock, sec = _loop_ensemble(ok, w, runs, steps, every, stream)
        t_total += sec
        rel = tr[:, :, 1] - tr[:, :, 0]
        case = {'x_rel_nm': w.extra['x_rel_nm'], 'z_rel_nm': w.extra['z_rel_nm']}
        case.update(_trajectory_summary(tr, clock))
        case.update({'x_rel_final_mean_nm': float(rel[:, -1].mean()),
                     'x_rel_final_min_max_nm': [float(rel[:, -1].min()), float(rel[:, -1].max())]})
        cases.append(case)
    out = {'metric': 'two-loop kinetics, loop coordinates along [111] against time', 'unit': 'nm',
           'data': 'synthetic', 'dtype': 'f32 fields / f64 energies',
           'config': {'workload': 'kinetics_two_loops_%dcubed (1/2<111> loops R = 3.3 nm, E_m = 0.1 eV, 300 K, '
                                  'Table 1 constants, 500 fixed-dt steps, 10 runs per case)' % args.box},
           'cases': cases, 'seconds': t_total, 'clocks': clk.stop()}
    print(json.dumps(out))
    return 0


def run_dislocation(args):
    """Loops near the paper's straight edge dislocation (line along [-1-12] through the
    box centre, b = (a0/2)[111]; Secs. 4.1, 4.3 and 5.2), 256^3, Table 1 constants.
    (1) The interaction energy of one loop (R = 3.3 nm, 4.85 nm from the line along
    [1-10]) with the dislocation against its position along [111], exact and in the
    dipole approximation, and of a <110> dumbbell SIA (Table 1's dipole tensor) on the
    same line.  (2) Two loops on both sides of the line (z = -/+4.85 nm),
    x_rel = 9.9 nm, centre of mass 20 or 30 nm from the line: 500 fixed-time-step steps
    at 300 K, 10 runs per case, the loops' coordinates along [111] against time."""
    import torch

    from paper_2403_09158_gb300 import okmc as ok
    from paper_2403_09158_gb300.workload import config_dislocation_loops

    stream = torch.cuda.current_stream()
    clk = Clocks(torch.cuda.current_device())
    w = config_dislocation_loops(20.0, n=args.box)
    lines = w.extra['lines']
    # (1) energy profile of loop 2 alone
    g = ok.Grid(w.n, w.voxel_nm, *w.C, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    g.set_dislocations(lines)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    one = w.defects[1:2].copy()
    z_site = one['pos'][0] - (one['pos'][0] @ np.ones(3) - 3 * w.n[0]) // 3   # the site at x = 0 on loop 2's z line
    one['pos'][0] = z_site
    g.set_defects(one)
    unit = 0.5 * w.voxel_nm
    profile = []
    for k in range(-100, 101, 4):
        pos = (z_site + k).reshape(1, 3).astype(np.int32)
        g.set_positions(pos)
        E = float(g.interaction_energies()[0])
        Ed = float(g.dipole_energies()[0][0])
        x = float(((pos[0] - np.array(w.n)) @ np.ones(3)) * unit / math.sqrt(3.0))
        profile.append([x, E, Ed])
    g.close()
    # (1b) Sec. 4.1: a <110> dumbbell SIA (dipole tensor of Table 1) probing the line's
    # field alone on the same z line
    g = ok.Grid(w.n, w.voxel_nm, *w.C, stream=stream.cuda_stream)
    g.set_dislocations(lines)
    P_sia = np.array([25.832, 21.143, 21.150, 5.122, 0.0, 0.0])       # Table 1, (xx, yy, zz, yz, xz, xy)
    ks = np.arange(-100, 101, 4)
    probes = (z_site[None, :] + ks[:, None]).astype(np.int32)
    E_sia = g.point_dipole_energies(probes, P_sia)
    profile_sia = [[float(k * unit * math.sqrt(3.0)), float(e)] for k, e in zip(ks, E_sia)]
    g.close()
    # (2) two-loop kinetics beside the line
    cases = []
    t_total = 0.0
    for x_c in (20.0, 30.0):
        wc = config_dislocation_loops(x_c, n=args.box)
        tr, clock, sec = _loop_ensemble(ok, wc, 10, 500, 10, stream, lines=lines)
        t_total += sec
        case = {'x_c_nm': x_c, 'x_nm': wc.extra['x_nm'], 'z_nm': wc.extra['z_nm']}
        case.update(_trajectory_summary(tr, clock))
        cases.append(case)
    out = {'metric': 'loops near an edge dislocation: energy profile and kinetics along [111]', 'unit': 'eV, nm',
           'data': 'synthetic', 'dtype': 'f32 fields / f64 energies',
           'config': {'workload': 'dislocation_two_loops_%dcubed (edge dislocation [-1-12], b = a0/2 [111]; '
                                  '1/2<111> loops R = 3.3 nm, E_m = 0.1 eV, 300 K, Table 1 constants)' % args.box},
           'setup_seconds': t_setup, 'profile_x_E_Edipole': profile, 'profile_sia_x_E': profile_sia,
           'cases': cases, 'seconds': t_total,
           'clocks': clk.stop()}
    print(json.dumps(out))
    return 0


def run_config(args, which):
    """The small (32^3, FP64 fields) and medium (128^3, FP32 fields beside the FP64 GPU
    path) workloads: residence-time steps per second and the latency of one
    request-level solve through the C ABI (move one defect from the host, then the
    stress solve and the site energies copied back)."""
    import torch

    from paper_2403_09158_gb300 import okmc as ok
    from paper_2403_09158_gb300.workload import config_medium, config_small

    w = config_small() if which == 'small' else config_medium()
    stream = torch.cuda.current_stream()
    N = int(np.prod(w.n))
    precs = [('f64', ok.FP64_FIELDS)] if which == 'small' else [('f32', ok.FP32_FIELDS), ('f64', ok.FP64_FIELDS)]
    out_paths = {}
    clk = Clocks(torch.cuda.current_device())
    for tag, prec in precs:
        g = ok.Grid(w.n, w.voxel_nm, *w.C, precision=prec, seed=w.seed, stream=stream.cuda_stream)
        g.set_defects(w.defects)
        for _ in range(args.warmup):
            g.step(w.T_K, 1)
        ms, events = _time_steps(g, w.T_K, args.steps, stream)
        # request-level solve latency: one defect moves (host positions in), then the
        # solve and the site energies (host array out)
        pos = g.get_positions()
        moved = pos.copy()
        E = np.zeros(g.nd)
        lat = []
        for k in range(max(5, args.steps // 2)):
            moved[:] = pos
            j = int(np.flatnonzero(w.defects['mobility'] != 0)[k % int((w.defects['mobility'] != 0).sum())])
            moved[j] = (moved[j] + (1 if k % 2 == 0 else -1)) % (2 * np.asarray(w.n))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.set_positions(moved)
            g.interaction_energies(E)
            lat.append(time.perf_counter() - t0)
        g.set_positions(pos)
        g.close()
        out_paths[tag] = {'ms_per_step': ms / args.steps, 'voxel_updates_per_s': N * args.steps / (ms / 1e3),
                          'events_per_s': events / (ms / 1e3), 'steps_per_s': args.steps / (ms / 1e3),
                          'solve_latency_ms_p50': float(np.percentile(np.array(lat) * 1e3, 50)),
                          'solve_latency_ms_max': float(max(lat) * 1e3)}
    clocks = clk.stop()
    head = out_paths[precs[0][0]]
    desc = ('small_32cubed (32^3, 2 1/2<111> loops R = 1 nm + 8 SIA clusters, 300 K, FP64 fields)' if which == 'small'
            else 'medium_128cubed_200defects (128^3, 200 defects, config-2 mix, 400 K)')
    out = {'metric': 'voxel stress+energy updates/s', 'value': head['voxel_updates_per_s'], 'unit': 'voxel updates/s',
           'n_gpus': 1, 'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': head['ms_per_step'],
           'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None,
           'dtype': 'f64' if which == 'small' else 'f32 fields / f64 energies', 'data': 'synthetic',
           'config': {'workload': desc, 'grid': list(w.n), 'defects': len(w.defects), 'mode': 'residence'},
           'paths': out_paths, 'clocks': clocks}
    print(json.dumps(out))
    return 0


def run_batch(args):
    """Ensemble of 64 independent replicas (edges 64-192, 50-800 defects capped by box
    volume, 300-600 K) advanced together: one CUDA graph launch per step, in the
    batched-kernel form (persistent kernels over work lists of every replica) and in
    the graph-branch form.  Compared with the same replicas stepped one after another
    (FP32) and with the single-replica FP64 path."""
    import torch

    from paper_2403_09158_gb300 import okmc as ok
    from paper_2403_09158_gb300.workload import config_batch

    ws = config_batch()
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    grids = []
    for w in ws:
        g = ok.Grid(w.n, w.voxel_nm, *w.C, precision=ok.FP32_FIELDS, seed=w.seed, stream=stream.cuda_stream)
        g.set_defects(w.defects)
        grids.append(g)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    voxels = sum(int(np.prod(w.n)) for w in ws)
    Ts = [w.T_K for w in ws]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clk = Clocks(torch.cuda.current_device())
    forms = {}
    for form in (ok.BATCH_KERNELS, ok.BATCH_GRAPHS):
        b = ok.Batch(grids, stream=stream.cuda_stream, mode=form)
        b.step(Ts, args.warmup)
        torch.cuda.synchronize()
        ev0 = sum(g.stats()['events'] for g in grids)
        e0.record(stream)
        b.step(Ts, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        forms[form] = (e0.elapsed_time(e1), sum(g.stats()['events'] for g in grids) - ev0, b.mode())
        b.close()
    clocks = clk.stop()
    ms, events, used = forms[ok.BATCH_KERNELS]
    ms_graph = forms[ok.BATCH_GRAPHS][0]
    # the same replicas one after another, each with its own step graph
    for g, T in zip(grids, Ts):
        g.step(T, 1)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(max(1, args.steps // 4)):
        for g, T in zip(grids, Ts):
            g.step(T, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    seq32_ms = e0.elapsed_time(e1) / max(1, args.steps // 4)
    for g in grids:
        g.close()
    # single-replica FP64 path: one replica per edge, timed alone, summed over the ensemble
    fp64_ms = {}
    for n in sorted({w.n[0] for w in ws}):
        w = next(x for x in ws if x.n[0] == n)
        g = ok.Grid(w.n, w.voxel_nm, *w.C, precision=ok.FP64_FIELDS, seed=w.seed, stream=stream.cuda_stream)
        g.set_defects(w.defects)
        g.step(w.T_K, 2)
        torch.cuda.synchronize()
        e0.record(stream)
        g.step(w.T_K, 5)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_ms[n] = e0.elapsed_time(e1) / 5
        g.close()
    seq64_ms = sum(fp64_ms[w.n[0]] for w in ws)
    value = voxels * args.steps / (ms / 1e3)
    out = {'metric': 'ensemble voxel stress+energy updates/s', 'value': value, 'unit': 'voxel updates/s', 'n_gpus': 1,
           'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': ms / args.steps, 'higher_is_better': True,
           'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f32 fields / f64 energies', 'data': 'synthetic',
           'config': {'workload': 'ensemble of 64 replicas (edge ~ U{64,96,128,160,192}, 50-800 defects capped by '
                                  'box volume, config-2 mix, T ~ U(300,600) K, residence-time steps)',
                      'voxels': voxels, 'defects': sum(len(w.defects) for w in ws),
                      'l2': 'inputs larger than L2 (%.1f GB of fields)' % (voxels * 16 / 1e9)},
           'events_per_s': events / (ms / 1e3), 'setup_s': setup_s,
           'form': 'batched persistent kernels: per edge class one branch of the three solve passes over '
                   'work lists of (replica, plane / tile) items, then energies, event and field update over every '
                   'replica; %d launches per step' % (3 * len({w.n for w in ws}) + 4),
           'graph_branches_fp32': {'ms_per_step': ms_graph / args.steps, 'value': voxels * args.steps / (ms_graph / 1e3),
                                   'note': 'each replica\'s own step as a branch of one graph (the other batch form)'},
           'sequential_fp32': {'ms_per_step': seq32_ms, 'value': voxels / (seq32_ms / 1e3)},
           'single_replica_fp64': {'ms_per_step_by_edge': fp64_ms, 'ms_per_ensemble_step': seq64_ms,
                                   'value': voxels / (seq64_ms / 1e3)},
           'vs_single_replica_fp64': (voxels / (ms / args.steps / 1e3)) / (voxels / (seq64_ms / 1e3)),
           'gpu_launches': (3 * len({w.n for w in ws}) + 4) * args.steps, 'clocks': clocks}
    print(json.dumps(out))
    return 0


def run_serve(args):
    """Serving: a pool of 32 resident replicas (edges 48-320) behind the request server
    (4 lanes, 120 GB admission budget); Poisson request streams at each offered rate,
    half solves (stress + site energies) and half steps of 1-10 events.  Latency is
    completion minus submission on the server's clock."""
    import torch

    from paper_2403_09158_gb300 import okmc as ok
    from paper_2403_09158_gb300.workload import config_serve, request_stream

    pool = config_serve()
    budget = 120 * 10 ** 9
    srv = ok.Server(hbm_budget=budget, lanes=4)
    ids = [srv.add_replica(w.n, w.voxel_nm, *w.C, w.defects, seed=w.seed) for w in pool]
    vox = [int(np.prod(w.n)) for w in pool]
    # admission of every replica (cold start), measured on its own
    t0 = time.perf_counter()
    cold = [srv.submit_solve(i) for i in ids]
    cold_lat = []
    solves = {}  # per replica: solves done so far (the work of a request is the solves it ran)
    for r, t in enumerate(cold):
        res, _ = srv.wait(t)
        assert res['status'] == 0, res
        cold_lat.append(res['t_end'] - res['t_submit'])
        solves[r] = res['stats']['solves']
    cold_s = time.perf_counter() - t0
    rates = [float(x) for x in args.rates.split(',')]
    per_rate = []
    clk = Clocks(torch.cuda.current_device())
    for k, rate in enumerate(rates):
        n_req = int(min(args.max_requests, max(40, rate * args.seconds)))
        reqs = request_stream(1005 + k, rate, n_req, len(ids))
        tickets = []
        start = time.perf_counter()
        for (ta, r, kind, kk) in reqs:
            while True:
                dt = start + ta - time.perf_counter()
                if dt <= 0:
                    break
                time.sleep(min(dt, 0.002))
            if kind == 'solve':
                tickets.append((srv.submit_solve(ids[r]), r))
            else:
                tickets.append((srv.submit_step(ids[r], pool[r].T_K, kk, positions=True), r))
        lat, t_first, t_last, work = [], None, None, 0
        for t, r in tickets:  # one replica's requests complete in submission order
            res, _ = srv.wait(t)
            assert res['status'] == 0, res
            lat.append(res['t_end'] - res['t_submit'])
            t_first = res['t_submit'] if t_first is None else min(t_first, res['t_submit'])
            t_last = res['t_end'] if t_last is None else max(t_last, res['t_end'])
            work += vox[r] * (res['stats']['solves'] - solves[r])
            solves[r] = res['stats']['solves']
        span = t_last - t_first
        lat = np.array(lat) * 1e3
        per_rate.append({'offered_req_per_s': rate, 'requests': n_req, 'achieved_req_per_s': n_req / span,
                         'voxel_updates_per_s': work / span, 'p50_ms': float(np.percentile(lat, 50)),
                         'p99_ms': float(np.percentile(lat, 99)), 'max_ms': float(lat.max())})
    clocks = clk.stop()
    st = srv.stats()
    srv.close()
    best = max(per_rate, key=lambda x: x['voxel_updates_per_s'])
    out = {'metric': 'served voxel stress+energy updates/s', 'value': best['voxel_updates_per_s'],
           'unit': 'voxel updates/s', 'n_gpus': 1, 'steps': None, 'warmup': None, 'higher_is_better': True,
           'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f32 fields / f64 energies', 'data': 'synthetic',
           'config': {'workload': 'serving: 32 replicas (edge ~ U{48,64,128,256,320}, 20-3000 defects capped at the '
                                  '256^3 density), Poisson arrivals, half solves and half steps of 1-10 events, '
                                  '4 lanes, 120 GB admission budget',
                      'replica_voxels': int(sum(vox)), 'defects': int(sum(len(w.defects) for w in pool))},
           'rates': per_rate, 'cold_start': {'seconds': cold_s, 'p50_ms': float(np.percentile(cold_lat, 50) * 1e3),
                                              'max_ms': float(max(cold_lat) * 1e3)},
           'server': st, 'clocks': clocks}
    print(json.dumps(out))
    return 0


class CpuStep:
    """The oracle as it stands doing the step of the 256^3 workload on a bounded sample:
    a 64^3 grid at the same defect density and mix (31 defects).  One step is what one
    GPU step does: voxelise every defect, one FP64 stress solve, the site and eight
    candidate energies of every defect (stencil sums over the stress minus the self
    terms), rates, one residence-time event.  The self terms are tabulated at set-up by
    the oracle's real-space route, as the GPU path tabulates them at okmc_set_defects;
    set-up is not part of a step."""

    def __init__(self):
        import oracle as O
        from paper_2403_09158_gb300.workload import scaled_population
        self.O = O
        w = scaled_population((64, 64, 64), 31, seed=77, T_K=500.0)
        self.w = w
        self.defs = w.defects.copy()
        self.C = O.stiffness_cubic(*w.C)
        t0 = time.perf_counter()
        kernels = {}
        self.W = []
        for d in self.defs:
            E, s = O.unit_tensor(d, w.voxel_nm)
            key = tuple(np.round(E.ravel(), 12))
            if key not in kernels:
                kernels[key] = O.unit_kernel(E, w.n, w.voxel_nm, self.C)
            self.W.append(O.self_term_table_realspace(d, w.n, w.voxel_nm, kernels[key], s))
        self.setup_s = time.perf_counter() - t0
        self.k = 0

    def step(self):
        O, w, h = self.O, self.w, self.w.voxel_nm
        t0 = time.perf_counter()
        sig = O.solve_stress(O.eigenstrain_field(self.defs, w.n, h), self.C, h)
        E = np.zeros(len(self.defs))
        Ec = np.zeros((len(self.defs), 8))
        for i, d in enumerate(self.defs):
            c = O.pos_class(d['pos'])
            E[i] = O.energy_of_stencil(d, d['pos'], sig, h) - self.W[i][c, 0]
            for j, Y in enumerate(O.candidate_positions(d['pos'])):
                Ec[i, j] = O.energy_of_stencil(d, Y, sig, h) - self.W[i][c, 1 + j]
        O.residence_step(self.defs, E, Ec, w.T_K, 77, self.k, w.n)
        self.k += 1
        return time.perf_counter() - t0

    SAMPLE = ('one residence step of the oracle on a 64^3 grid at the 256^3 workload\'s density and mix (31 '
              'defects): voxelise, FP64 stress solve, site + 8 candidate energies of every defect (stencil sums '
              'minus self terms tabulated at set-up by the oracle\'s real-space route, not timed), rates, one '
              'event; numpy, 1 thread')


def cpu_sample():
    """One timed oracle step after set-up (see CpuStep)."""
    cs = CpuStep()
    dt = cs.step()
    return dict(value=64 ** 3 / dt, seconds=dt, cores=1, host_cores=os.cpu_count(), setup_s=cs.setup_s,
                sample=CpuStep.SAMPLE)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=30)
    ap.add_argument('--warmup', type=int, default=5)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--workload', default='large', choices=['large', 'batch', 'serve', 'small', 'medium', 'dipole',
                                                            'kinetics', 'dislocation'],
                    help='large: the 256^3 single-replica step (default); batch: the 64-replica ensemble; '
                         'serve: the request server under Poisson load; small / medium: the 32^3 FP64 and '
                         'the 128^3 workloads')
    ap.add_argument('--box', type=int, default=256, help='kinetics, dislocation: box edge in voxels (512 is close to the '
                                                          "paper's 500 a0)")
    ap.add_argument('--rates', default='10,30,100,300,1000,2000', help='serve: offered request rates (1/s)')
    ap.add_argument('--seconds', type=float, default=4.0, help='serve: length of each rate\'s request stream')
    ap.add_argument('--max-requests', type=int, default=600, help='serve: cap on requests per rate')
    ap.add_argument('--solve-only', type=int, default=0, metavar='N',
                    help='profiling aid: one stress solve of an N^3 grid holding one SIA cluster, then exit')
    args = ap.parse_args()
    ws, rank = _dist()
    if args.solve_only:
        return solve_only(args.solve_only)
    if args.impl == 'reference':
        return run_reference(args, ws, rank)
    import torch
    if ws > 1:
        torch.distributed.init_process_group('nccl' if torch.cuda.is_available() else 'gloo')
    import __graft_entry__
    __graft_entry__.build()
    if args.workload == 'batch':
        return run_batch(args) if rank == 0 else 0
    if args.workload == 'serve':
        return run_serve(args) if rank == 0 else 0
    if args.workload in ('small', 'medium'):
        return run_config(args, args.workload) if rank == 0 else 0
    if args.workload == 'dipole':
        return run_dipole(args) if rank == 0 else 0
    if args.workload == 'kinetics':
        return run_kinetics(args) if rank == 0 else 0
    if args.workload == 'dislocation':
        return run_dislocation(args) if rank == 0 else 0
    r = run_ours(args, ws, rank)
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return 0
    steps = args.steps
    value = ws * r['N'] * steps / (r['ms'] / 1e3)
    hbm, src = _peaks()
    kt = r['kt']
    dom = max((k for k in kt if kernel_bytes(k, r['n'])), key=lambda k: kt[k][0])
    d_ms, d_cnt = kt[dom]
    achieved = kernel_bytes(dom, r['n']) / (d_ms / d_cnt / 1e3) / 1e9
    solve_ms = sum(kt[k][0] for k in ('plane_fwd', 'pencil_green', 'plane_inv') if k in kt) / max(1, kt.get('plane_fwd', (0, 1))[1])
    pipe_gbs = 96 * r['N'] / (solve_ms / 1e3) / 1e9
    launches = sum(c for (_, c) in kt.values())  # the same kernels per step in both timed regions
    full_k = {k: float(np.median([f[k] for f in r['full'] if k in f])) for k in ('plane_fwd', 'pencil_green', 'plane_inv')}
    full_ms = sum(full_k.values())
    out = {
        'metric': METRIC, 'value': value, 'unit': UNIT, 'n_gpus': ws, 'steps': steps, 'warmup': args.warmup,
        'ms_per_step': r['ms'] / steps, 'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None,
        'dtype': 'f32 fields / f64 energies', 'data': 'synthetic',
        'config': {'workload': 'large_256cubed_2000defects (256^3 voxels, h=0.2855 nm, 2000 defects: 60% SIA clusters, '
                               '30% 1/2<111> loops, 10% <100> loops, R~U(0.5,4) nm, 500 K, residence-time steps)',
                   'grid': list(r['n']), 'defects': r['nd'], 'mode': 'residence',
                   'l2': 'inputs larger than L2 (6-component fields of 403 MB each)', 'parallelism': 'replicas'},
        'events_per_s': ws * r['events'] / (r['ms'] / 1e3),
        'setup_s': r['setup_s'],
        'roofline': {'bound': 'hbm', 'kernel': dom, 'achieved': achieved, 'peak': hbm, 'unit': 'GB/s',
                     'frac': achieved / hbm, 'traffic': measured_traffic(dom),
                     'algorithmic_bytes': kernel_bytes(dom, r['n']), 'peak_source': src + ' copy bandwidth',
                     'timing': 'CUDA events around each launch on the handle stream, over a second timed region '
                               'of the same number of steps'},
        'pipeline_roofline': {'kind': 'incremental step: the forward plane pass transforms only the planes '
                                      'whose eigenstrain changed (exact, bitwise equal to a full pass)',
                              'solve_ms': solve_ms, 'algorithmic_bytes': 96 * r['N'], 'achieved_gbs': pipe_gbs,
                              'frac': pipe_gbs / hbm},
        'full_solve_ms': full_ms, 'full_solve_frac': 96 * r['N'] / (full_ms / 1e3) / 1e9 / hbm,
        'full_solve': {'kernel_ms': full_k, 'algorithmic_bytes': 96 * r['N'],
                       'moved_bytes_three_pass': 144 * r['N'],
                       'moved_frac': 144 * r['N'] / (full_ms / 1e3) / 1e9 / hbm,
                       'note': 'every plane dirty (after okmc_set_defects); B_alg = 96 N, the three-pass design '
                               'moves 144 N (the pencil pass reads and writes the spectrum once more)'},
        'latency_ms': {'p50': float(np.percentile(r['lat_ms'], 50)), 'p99': float(np.percentile(r['lat_ms'], 99)),
                       'requests': len(r['lat_ms']),
                       'request': 'one step end to end through the C ABI: positions in from pinned host memory, '
                                  'step, positions and statistics out (host clock)'},
        'repeats': {'count': len(r['repeats']),
                    'ms_per_step_median': float(np.median(r['repeats'])) / steps if r['repeats'] else None,
                    'ms_per_step_min': float(np.min(r['repeats'])) / steps if r['repeats'] else None,
                    'ms_per_step_max': float(np.max(r['repeats'])) / steps if r['repeats'] else None,
                    'note': 'the K-step region repeated for about a second inside the clock record'},
        'kernel_ms': {k: v[0] / v[1] for k, v in kt.items()},
        'cufft_reference': {'fwd_inv_ms': r['cufft'], 'solve_ms': solve_ms,
                            'note': 'torch.fft (cuFFT) R2C + C2R of the six components on the same grid, no Green '
                                    'operator, on fresh input (no clean-plane reuse); solve_ms is the three solve '
                                    'kernels of one step here'},
        'gpu_launches': int(launches),
        'clocks': r['clocks'],
        'e2e': {'value': ws * r['N'] / r['e2e_s'], 'unit': UNIT, 'h2d_bytes_per_step': r['nd'] * 12,
                'd2h_bytes_per_step': r['nd'] * 12 + r['stats_bytes']},
    }
    if not args.no_cpu_baseline:
        cb = cpu_sample()
        out['cpu_baseline'] = {'value': cb['value'], 'unit': UNIT, 'cores': cb['cores'], 'host_cores': cb['host_cores'],
                               'kind': 'oracle', 'sample': cb['sample'], 'setup_s': cb['setup_s'],
                               'step_s': cb['seconds']}
    print(json.dumps(out))
    return 0


def solve_only(n):
    """Launch sequence: self-term build (plane_fwd, pencil forward), then one solve
    (plane_fwd, pencil_green, plane_inv)."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_09158_gb300 import okmc as ok
    from paper_2403_09158_gb300.workload import make_defects
    g = ok.Grid((n, n, n), 0.2855, 243.0, 145.0, 116.0)
    g.set_defects(make_defects([2], np.array([[1, 1, 1]]), [0], [0.0], [3], [0.3], [2]))
    g.solve_stress(copy=False)
    g.close()
    print(json.dumps({'solve_only': n}))
    return 0


# the source files that hold each timed kernel's device code
KERNEL_SOURCES = {
    'plane_fwd': ('solve_fast.cu', 'fft_reg.cuh', 'okmc_internal.cuh'),
    'pencil_green': ('solve_fast.cu', 'fft_reg.cuh', 'okmc_internal.cuh'),
    'plane_inv': ('solve_fast.cu', 'fft_reg.cuh', 'okmc_internal.cuh'),
    'energies': ('defects.cu', 'okmc_internal.cuh'),
}


def kernel_sources_hash(kernel):
    """Hash of the files that hold `kernel`'s device code (a change elsewhere, e.g. in
    the C ABI layer or another kernel's file, does not change its DRAM traffic)."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, 'paper_2403_09158_gb300', 'csrc')
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(d, f), 'rb').read())
    return h.hexdigest()[:16]


def measured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from profiles/dram_traffic.json, if that capture
    was taken on the kernel's current sources (else None)."""
    p = os.path.join(ROOT, 'profiles', 'dram_traffic.json')
    if not os.path.exists(p) or kernel not in KERNEL_SOURCES:
        return None
    k = json.load(open(p)).get('kernels', {}).get(kernel)
    if k is None or k.get('sources_hash') != kernel_sources_hash(kernel):
        return None
    return k.get('dram_bytes_per_launch')


def run_reference(args, ws, rank):
    """The CPU FP64 oracle as the reference arm, on this arm's metric and unit: set-up
    once (not timed), W warm-up steps, then K timed steps of CpuStep."""
    if rank != 0:
        return 0
    cs = CpuStep()
    for _ in range(args.warmup):
        cs.step()
    times = [cs.step() for _ in range(args.steps)]
    per = float(np.mean(times))
    value = 64 ** 3 / per
    out = {'impl': 'reference', 'metric': METRIC, 'value': value, 'unit': UNIT, 'n_gpus': 1, 'steps': args.steps,
           'warmup': args.warmup, 'ms_per_step': per * 1e3, 'higher_is_better': True, 'scaling': 'weak',
           'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
           'config': {'workload': 'large_256cubed_2000defects, sampled as a 64^3 grid at the same defect density'},
           'cpu_baseline': {'value': value, 'unit': UNIT, 'cores': 1, 'host_cores': os.cpu_count(), 'kind': 'oracle',
                            'sample': CpuStep.SAMPLE, 'setup_s': cs.setup_s},
           'e2e': {'value': value, 'unit': UNIT, 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}}
    print(json.dumps(out))
    return 0


if __name__ == '__main__':
    sys.exit(main())
