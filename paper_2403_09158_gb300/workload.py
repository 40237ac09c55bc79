"""Seeded synthetic workloads: defect lists in the paper's setting.

Only random draws and placement live here (no eigenstrain, solve, energy or
rate arithmetic), so that the CUDA path and the CPU oracle can be fed the very
same inputs.  Defect mix, sizes and temperatures follow the paper's OkMC
setting for bcc Fe (Sec. 5: 1/2<111> loops migrating in 1D with E_m = 0.1 eV,
<100> loops immobile, SIAs migrating in 3D; Sec. 5.3: ~6e18 cm^-3 SIA density).

Records use ``DEFECT_DTYPE``, whose memory layout is the C struct
``okmc_defect`` of ``include/okmc.h`` (48 bytes, little endian).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LOOP_111, LOOP_100, SIA_CLUSTER = 0, 1, 2
IMMOBILE, ONE_D, THREE_D = 0, 1, 2

DEFECT_DTYPE = np.dtype([
    ('type', '<i4'), ('pos', '<i4', (3,)), ('axis', '<i4'), ('size', '<i4'),
    ('mobility', '<i4'), ('reserved', '<i4'), ('radius_nm', '<f8'), ('Em_eV', '<f8'),
])
assert DEFECT_DTYPE.itemsize == 48

FE_CUBIC = (243.0, 145.0, 116.0)         # C11, C12, C44 in GPa (synthetic Fe constants)
FE_ISO = (82.0, 0.29)                    # mu (GPa), nu
FE_TABLE1 = (289.34, 152.34, 107.43)     # Table 1 of the paper
VOXEL_NM = 0.2855                        # a0 = voxel edge h


@dataclass
class Workload:
    name: str
    n: tuple
    voxel_nm: float
    defects: np.ndarray
    T_K: float
    C: tuple = FE_CUBIC
    seed: int = 0
    events: int = 0
    extra: dict = field(default_factory=dict)


def _shape_radius_nm(kind, radius_nm, size, h):
    if kind == SIA_CLUSTER:
        return max(h, (3.0 * size * 0.5 * h ** 3 / (4.0 * math.pi)) ** (1.0 / 3.0))
    return radius_nm


def place(rng, n, h, kinds, radii, sizes, max_tries=20000):
    """Uniform bcc sites (integer half-lattice coordinates, all even or all odd),
    rejecting a site closer than R_i + R_j + 2h (minimum image) to an earlier one."""
    n = np.asarray(n)
    L = n * h
    m = len(kinds)
    pos = np.zeros((m, 3), dtype=np.int64)
    centres = np.zeros((m, 3))
    rr = np.zeros(m)
    for i, (k, R, s) in enumerate(zip(kinds, radii, sizes)):
        Ri = _shape_radius_nm(k, R, s, h)
        for _ in range(max_tries):
            c = int(rng.integers(0, 2))
            p = 2 * rng.integers(0, n) + c
            x = p * (h / 2.0)
            dvec = x - centres[:i]
            dvec -= L * np.round(dvec / L)
            if not np.any(np.sqrt(np.einsum('ij,ij->i', dvec, dvec)) < Ri + rr[:i] + 2.0 * h):
                break
        else:
            raise RuntimeError('could not place defect %d' % i)
        pos[i] = p
        centres[i] = x
        rr[i] = Ri
    return pos


def make_defects(kinds, pos, axes, radii, sizes, Em, mobility):
    d = np.zeros(len(kinds), dtype=DEFECT_DTYPE)
    d['type'] = kinds
    d['pos'] = pos
    d['axis'] = axes
    d['radius_nm'] = radii
    d['size'] = sizes
    d['Em_eV'] = Em
    d['mobility'] = mobility
    return d


def mixed_population(n, n_defects, seed, frac=(0.6, 0.3, 0.1), r111=(0.5, 2.5),
                     r100=(1.0, 3.0), p_geom=0.3, h=VOXEL_NM, single_sia_3d=True,
                     em_loop=0.1, em_sia=0.3):
    """SIA clusters (size ~ Geometric(p)), 1/2<111> loops and <100> loops in the given
    fractions, uniform positions and orientations."""
    rng = np.random.default_rng(seed)
    n_sia = int(round(frac[0] * n_defects))
    n_111 = int(round(frac[1] * n_defects))
    n_100 = n_defects - n_sia - n_111
    kinds = np.array([SIA_CLUSTER] * n_sia + [LOOP_111] * n_111 + [LOOP_100] * n_100)
    sizes = np.zeros(n_defects, dtype=np.int64)
    sizes[:n_sia] = rng.geometric(p_geom, n_sia)
    radii = np.zeros(n_defects)
    radii[n_sia:n_sia + n_111] = rng.uniform(r111[0], r111[1], n_111)
    radii[n_sia + n_111:] = rng.uniform(r100[0], r100[1], n_100)
    axes = np.zeros(n_defects, dtype=np.int64)
    axes[:n_sia + n_111] = rng.integers(0, 4, n_sia + n_111)
    axes[n_sia + n_111:] = rng.integers(0, 3, n_100)
    # place large defects first so rejection sampling converges
    order = np.argsort(-np.array([_shape_radius_nm(k, r, s, h) for k, r, s in zip(kinds, radii, sizes)]),
                       kind='stable')
    pos_sorted = place(rng, n, h, kinds[order], radii[order], sizes[order])
    pos = np.zeros_like(pos_sorted)
    pos[order] = pos_sorted
    Em = np.where(kinds == SIA_CLUSTER, em_sia, np.where(kinds == LOOP_111, em_loop, 1.0))
    mob = np.where(kinds == LOOP_100, IMMOBILE, ONE_D)
    if single_sia_3d:
        mob = np.where((kinds == SIA_CLUSTER) & (sizes == 1), THREE_D, mob)
    return make_defects(kinds, pos, axes, radii, sizes, Em, mob)


def config_small(seed=1001, n=32, h=VOXEL_NM):
    """32^3 box: two 1/2[111] loops (R = 1 nm) at a seeded separation of 2-6 nm and
    8 SIA clusters of 1-10 atoms migrating in 1D (E_m = 0.3 eV); 300 K."""
    rng = np.random.default_rng(seed)
    L = n * h
    for _ in range(1000):
        sep = rng.uniform(2.0, 6.0)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        p0 = 2 * (np.array([n, n, n]) // 2)
        dp = np.round(u * sep / (h / 2.0)).astype(np.int64)
        if np.any((dp & 1) != (dp[0] & 1)):
            dp = 2 * np.round(u * sep / h).astype(np.int64)
        p1 = np.mod(p0 + dp, 2 * n)
        if 2.0 <= np.linalg.norm(dp * h / 2.0) <= 6.0 + h:
            break
    loops = make_defects([LOOP_111, LOOP_111], np.stack([p0, p1]), [0, 0], [1.0, 1.0], [0, 0],
                         [0.1, 0.1], [ONE_D, ONE_D])
    sizes = rng.integers(1, 11, 8)
    kinds = [SIA_CLUSTER] * 8
    occupied = [(p0 * h / 2.0, 1.0), (p1 * h / 2.0, 1.0)]
    pos = []
    for s in sizes:
        Ri = _shape_radius_nm(SIA_CLUSTER, 0.0, s, h)
        while True:
            c = int(rng.integers(0, 2))
            p = 2 * rng.integers(0, n, 3) + c
            x = p * h / 2.0
            ok = True
            for xc, Rj in occupied:
                dv = x - xc
                dv -= L * np.round(dv / L)
                if np.linalg.norm(dv) < Ri + Rj + 2.0 * h:
                    ok = False
                    break
            if ok:
                break
        occupied.append((x, Ri))
        pos.append(p)
    sias = make_defects(kinds, np.array(pos), rng.integers(0, 4, 8), np.zeros(8), sizes,
                        np.full(8, 0.3), np.full(8, ONE_D))
    d = np.concatenate([loops, sias])
    return Workload('small_32cubed_2loops_8sia', (n, n, n), h, d, 300.0, FE_CUBIC, seed, 100)


def config_medium(seed=1002, n=128, n_defects=200):
    """128^3 box, 200 defects: 60 % SIA clusters, 30 % 1/2<111> loops R ~ U(0.5, 2.5) nm,
    10 % <100> loops R ~ U(1, 3) nm; 400 K."""
    d = mixed_population((n, n, n), n_defects, seed, r111=(0.5, 2.5), r100=(1.0, 3.0))
    return Workload('medium_128cubed_200defects', (n, n, n), VOXEL_NM, d, 400.0, FE_CUBIC, seed, 10000)


def config_large(seed=1003, n=256, n_defects=2000):
    """256^3 box, 2000 defects with the same mix, all loop radii ~ U(0.5, 4) nm; 500 K."""
    d = mixed_population((n, n, n), n_defects, seed, r111=(0.5, 4.0), r100=(0.5, 4.0))
    return Workload('large_256cubed_2000defects', (n, n, n), VOXEL_NM, d, 500.0, FE_CUBIC, seed, 10000)


def scaled_population(n, n_defects, seed, T_K=500.0, r111=(0.5, 4.0), r100=(0.5, 4.0)):
    """Any grid with the large-config mix (used for ragged and intermediate sizes)."""
    n = tuple(int(v) for v in (n if np.ndim(n) else (n, n, n)))
    d = mixed_population(n, n_defects, seed, r111=r111, r100=r100)
    return Workload('mix_%dx%dx%d_%d' % (n + (n_defects,)), n, VOXEL_NM, d, T_K, FE_CUBIC, seed, 0)


def density_cap(n):
    """Largest defect count drawn for an n^3 box in the ensemble and serving workloads:
    150 per 64^3 box scaled by volume.  With the config-2 radii and the
    R_i + R_j + 2h exclusion of ``place``, larger counts do not fit a small box
    (64^3 with 300 defects already fails)."""
    return max(1, int(150 * (n / 64.0) ** 3))


def _placed_population(n, nd, seed, r111, r100):
    """mixed_population with the count lowered by 10 % until placement succeeds
    (deterministic for a given seed)."""
    while True:
        try:
            return mixed_population((n, n, n), nd, seed, r111=r111, r100=r100)
        except RuntimeError:
            if nd <= 1:
                raise
            nd = max(1, int(nd * 0.9))


def config_kinetics(x_rel_nm, n=256, h=VOXEL_NM, z_rel_nm=10.0, R_nm=3.3, T_K=300.0):
    """The paper's two-loop kinetics setting (Sec. 5.1): two 1/2<111> loops of radius
    3.3 nm (the loops of Sec. 4), Burgers vectors, normals and glide along [111] (the
    paper's x axis), separated by z_rel across the glide axis along [1-10] (the paper's
    z) and by x_rel along it; E_m = 0.1 eV, 300 K, the elastic constants of Table 1.
    Loop 1 sits at the box centre; both positions are bcc sites in units of a0/2."""
    unit = 0.5 * h                                   # a0/2 in nm
    kz = 2 * int(round(z_rel_nm / (unit * math.sqrt(2.0)) / 2.0))   # even: keeps the parity
    kx = int(round(x_rel_nm / (unit * math.sqrt(3.0))))
    c0 = np.array([n, n, n])
    p2 = c0 + np.array([kz, -kz, 0]) + kx
    defs = make_defects([LOOP_111, LOOP_111], np.array([c0, p2]), [0, 0], [R_nm, R_nm], [0, 0], [0.1, 0.1],
                        [ONE_D, ONE_D])
    return Workload(name='kinetics_two_loops_x%.0fA' % (10 * x_rel_nm), n=(n, n, n), voxel_nm=h, defects=defs,
                    T_K=T_K, C=FE_TABLE1,
                    extra={'x_rel_nm': kx * unit * math.sqrt(3.0), 'z_rel_nm': kz * unit * math.sqrt(2.0)})


def frame_111():
    """The paper's frame for loops and dislocations (Sec. 4): x = [111]/sqrt3 (Burgers
    vector and glide of the loops), y = [-1-12]/sqrt6, z = [1-10]/sqrt2, as cube-axis
    unit vectors."""
    return (np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0), np.array([-1.0, -1.0, 2.0]) / math.sqrt(6.0),
            np.array([1.0, -1.0, 0.0]) / math.sqrt(2.0))


def edge_dislocation_y(n, h):
    """One period of the paper's straight edge dislocation (Sec. 4.1): line along y =
    [-1-12] through the box centre, b = (a0/2)[111] along x.  In a cubic box of edge n h
    with cube-axis grid lines, the period is n (-1,-1,2) h (its end is a lattice
    translate of its start); the nearest periodic image lies n h / sqrt3 away."""
    c = 0.5 * np.asarray(n, float) * h
    d = np.array([-1.0, -1.0, 2.0]) * (0.5 * n[0] * h)
    return [(np.array([c - d, c + d]), 0.5 * h * np.ones(3), False)]


def config_dislocation_loops(x_c_nm, n=256, h=VOXEL_NM, z_nm=5.0, x_rel_nm=10.0, R_nm=3.3, T_K=300.0):
    """The paper's two loops near an edge dislocation (Sec. 5.2): 1/2<111> loops (R =
    3.3 nm, E_m = 0.1 eV, 1D glide along x = [111]) on both sides of the line, z = -z_nm
    (loop 1) and +z_nm (loop 2) along [1-10], their centre of mass x_c_nm from the line
    along x and x_rel_nm apart (loop 1 behind).  Positions are the nearest bcc sites that
    keep the z offsets symmetric (even multiples of (1,-1,0) in a0/2 units)."""
    assert n % 2 == 0
    unit = 0.5 * h
    kz = 2 * int(round(z_nm / (unit * math.sqrt(2.0)) / 2.0))
    k1 = int(round((x_c_nm - 0.5 * x_rel_nm) / (unit * math.sqrt(3.0))))
    k2 = int(round((x_c_nm + 0.5 * x_rel_nm) / (unit * math.sqrt(3.0))))
    c0 = np.array([n, n, n])
    p1 = c0 + np.array([-kz, kz, 0]) + k1
    p2 = c0 + np.array([kz, -kz, 0]) + k2
    defs = make_defects([LOOP_111, LOOP_111], np.array([p1, p2]), [0, 0], [R_nm, R_nm], [0, 0], [0.1, 0.1],
                        [ONE_D, ONE_D])
    xs = [k * unit * math.sqrt(3.0) for k in (k1, k2)]
    return Workload(name='dislocation_two_loops_xc%.0fA' % (10 * x_c_nm), n=(n, n, n), voxel_nm=h, defects=defs,
                    T_K=T_K, C=FE_TABLE1,
                    extra={'lines': edge_dislocation_y((n, n, n), h), 'x_nm': xs, 'z_nm': [-kz * unit * math.sqrt(2.0),
                                                                                           kz * unit * math.sqrt(2.0)]})


def config_batch(seed=1004, n_replicas=64, edges=(64, 96, 128, 160, 192), nd_range=(50, 800),
                 T_range=(300.0, 600.0)):
    """Ensemble of independent replicas: edge ~ U(edges), defect count ~ U{50..800}
    capped by ``density_cap``, config-2 mix and radii, T ~ U(300, 600) K."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_replicas):
        n = int(rng.choice(edges))
        nd = min(int(rng.integers(nd_range[0], nd_range[1] + 1)), density_cap(n))
        T = float(rng.uniform(*T_range))
        d = _placed_population(n, nd, seed * 1000 + r, (0.5, 2.5), (1.0, 3.0))
        out.append(Workload('replica%02d_%dcubed_%d' % (r, n, len(d)), (n, n, n), VOXEL_NM, d, T, FE_CUBIC,
                            seed * 1000 + r, 1000))
    return out


def config_serve(seed=1005, n_replicas=32, edges=(48, 64, 128, 256, 320), nd_range=(20, 3000),
                 T_range=(300.0, 600.0)):
    """Replica pool of the serving workload: edge ~ U(edges), defect count ~ U{20..3000}
    capped at the 256^3 workload's density (2000 per 256^3 box, at least 20), the
    large-config mix (loop radii U(0.5, 4) nm, at most a quarter of the box),
    T ~ U(300, 600) K."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_replicas):
        n = int(rng.choice(edges))
        cap = max(nd_range[0], int(2000 * (n / 256.0) ** 3))
        nd = min(int(rng.integers(nd_range[0], nd_range[1] + 1)), cap)
        T = float(rng.uniform(*T_range))
        rmax = min(4.0, 0.25 * n * VOXEL_NM)
        d = _placed_population(n, nd, seed * 1000 + r, (0.5, rmax), (0.5, rmax))
        out.append(Workload('serve%02d_%dcubed_%d' % (r, n, len(d)), (n, n, n), VOXEL_NM, d, T, FE_CUBIC,
                            seed * 1000 + r, 0))
    return out


def request_stream(seed, rate, n_requests, n_replicas, p_solve=0.5, k_range=(1, 10)):
    """Poisson arrivals at `rate` per second: (arrival time s, replica, kind, k) with kind
    'solve' or 'step' (k steps, k ~ U{1..10})."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    reqs = []
    for i in range(n_requests):
        r = int(rng.integers(0, n_replicas))
        if rng.random() < p_solve:
            reqs.append((float(t[i]), r, 'solve', 1))
        else:
            reqs.append((float(t[i]), r, 'step', int(rng.integers(k_range[0], k_range[1] + 1))))
    return reqs
