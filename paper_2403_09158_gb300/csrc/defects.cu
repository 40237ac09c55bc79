// Defect-side kernels: eigenstrain stencils (paper Sec. 3.1, Eq. eig_shearloop;
// Sec. 3.4 voxel grid), voxelisation, incremental position updates, the
// self-term table, interaction and candidate energies (Sec. 2, Eq.
// interaction_energy3), rates and event selection (Sec. 5, Eqs.
// unbiased_boltzmann, biased_forward/backward_boltzmann, frequency_line,
// selection_jump, time_step, poisson; Appendix A, Algorithm 1).
#include <cstdio>

#include "okmc_internal.cuh"

namespace okmc {

// ---------------------------------------------------------------- setup
// Geometry of one defect (a0 = h).  Loop: slab |(x-X).n| <= h/2 and in-plane
// radius <= R with n = a/|a|; eps* = sym(b (x) n)/h = (|b|/h) n (x) n.  SIA
// cluster of s atoms: sphere of radius h*max(1, (3 s / 8 pi)^(1/3)) (Omega =
// h^3/2) with dilatational eps* whose integral has trace 1.5 s Omega.
__global__ void k_defect_setup(const okmc_defect* __restrict__ d, DefGeo* __restrict__ G, int nd, double h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  const okmc_defect r = d[i];
  DefGeo g = {};
  if (r.type == OKMC_LOOP_111 || r.type == OKMC_LOOP_100) {
    int a[3];
    if (r.type == OKMC_LOOP_111) {
      a[0] = (r.axis == 1) ? -1 : 1;
      a[1] = (r.axis == 2) ? -1 : 1;
      a[2] = (r.axis == 3) ? -1 : 1;
    } else {
      a[0] = r.axis == 0;
      a[1] = r.axis == 1;
      a[2] = r.axis == 2;
    }
    const int a2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    const double bh = (r.type == OKMC_LOOP_111) ? 0.86602540378443864676 : 1.0;  // |b|/h
    const double f = bh / (double)a2;
    g.e6[0] = f * a[0] * a[0];
    g.e6[1] = f * a[1] * a[1];
    g.e6[2] = f * a[2] * a[2];
    g.e6[3] = f * a[1] * a[2];
    g.e6[4] = f * a[0] * a[2];
    g.e6[5] = f * a[0] * a[1];
    const double t = 8.0 * r.radius_nm / h;
    g.thr = (double)a2 * (t * t);
    const double rh = r.radius_nm / h;
    g.v_over_h3 = kPi * (rh * rh);
    g.kind = 0;
    g.a[0] = a[0];
    g.a[1] = a[1];
    g.a[2] = a[2];
    g.a2 = a2;
    g.extent = (int)ceil(rh) + 2;
  } else {
    const double q = 3.0 * r.size / (8.0 * kPi);
    const double rho3 = q > 1.0 ? q : 1.0;
    g.thr = 262144.0 * (rho3 * rho3);
    g.v_over_h3 = (4.0 * kPi / 3.0) * rho3;
    const double e = (1.5 * r.size * 0.5) / (3.0 * g.v_over_h3);
    g.e6[0] = g.e6[1] = g.e6[2] = e;
    g.kind = 1;
    g.extent = (int)ceil(cbrt(rho3)) + 2;
  }
  int mask = 0;
  if (r.mobility == OKMC_THREE_D) mask = 0xFF;
  if (r.mobility == OKMC_ONE_D) {
    const int sx = (r.axis == 1) ? -1 : 1, sy = (r.axis == 2) ? -1 : 1, sz = (r.axis == 3) ? -1 : 1;
    const int jp = 4 * (sx > 0) + 2 * (sy > 0) + (sz > 0);
    mask = (1 << jp) | (1 << (7 - jp));
  }
  g.allowed = mask;
  g.z = __popc(mask);
  g.escale = g.kind == 0 ? ((r.type == OKMC_LOOP_111) ? 0.86602540378443864676 : 1.0) / (double)g.a2 : g.e6[0];
  if (!(g.escale > 0.0)) g.escale = 1.0;
  for (int a = 0; a < 6; ++a) g.ew[a] = (float)((a < 3 ? 1.0 : 2.0) * g.e6[a] / g.escale);
  G[i] = g;
}

// subsample coordinates relative to the centre, in units of h/8: s = 8 v + 2 i + 1 - 4 c
__device__ __forceinline__ int coverage(const DefGeo& g, int c, int dx, int dy, int dz) {
  int cnt = 0;
  for (int i = 0; i < 4; ++i) {
    const int sx = 8 * dx + 2 * i + 1 - 4 * c;
    for (int j = 0; j < 4; ++j) {
      const int sy = 8 * dy + 2 * j + 1 - 4 * c;
      for (int l = 0; l < 4; ++l) {
        const int sz = 8 * dz + 2 * l + 1 - 4 * c;
        const long long ss = (long long)sx * sx + (long long)sy * sy + (long long)sz * sz;
        bool in;
        if (g.kind == 0) {
          const long long sa = (long long)g.a[0] * sx + (long long)g.a[1] * sy + (long long)g.a[2] * sz;
          in = (sa * sa <= 16ll * g.a2) && ((double)(g.a2 * ss - sa * sa) <= g.thr);
        } else {
          in = (double)(ss * ss * ss) <= g.thr;
        }
        cnt += in;
      }
    }
  }
  return cnt;
}

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < nw; ++k) t += sh[k];  // fixed order: deterministic
  __syncthreads();
  return t;
}

__device__ __forceinline__ long long block_sum_ll(long long v, long long* sh) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  long long t = 0;
  for (int k = 0; k < nw; ++k) t += sh[k];
  __syncthreads();
  return t;
}

// One block per (defect, class): number of stencil entries and total subsample count.
__global__ void k_stencil_count(const DefGeo* __restrict__ G, int* __restrict__ nnz, long long* __restrict__ sumcnt) {
  __shared__ long long sh[32];
  const int i = blockIdx.x >> 1, c = blockIdx.x & 1;
  const DefGeo g = G[i];
  const int E = g.extent, side = 2 * E + 1;
  const int nv = side * side * side;
  long long n = 0, s = 0;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const int dx = v % side - E, dy = (v / side) % side - E, dz = v / (side * side) - E;
    const int k = coverage(g, c, dx, dy, dz);
    n += (k > 0);
    s += k;
  }
  n = block_sum_ll(n, sh);
  s = block_sum_ll(s, sh);
  if (threadIdx.x == 0) {
    nnz[blockIdx.x] = (int)n;
    sumcnt[blockIdx.x] = s;
  }
}

// One block per (defect, class): entries in (dz, dy, dx) order; alpha = V/(h^3 sum count).
__global__ void k_stencil_fill(const DefGeo* __restrict__ G, const int* __restrict__ ptr,
                               const long long* __restrict__ sumcnt, int* __restrict__ off,
                               uint8_t* __restrict__ cnt, double* __restrict__ alpha, int* __restrict__ err) {
  __shared__ int wsum[32];
  __shared__ int base_s;
  const int i = blockIdx.x >> 1, c = blockIdx.x & 1;
  const DefGeo g = G[i];
  const int E = g.extent, side = 2 * E + 1;
  const int nv = side * side * side;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base_s = ptr[blockIdx.x];
  __syncthreads();
  for (int v0 = 0; v0 < nv; v0 += blockDim.x) {
    const int v = v0 + threadIdx.x;
    int k = 0, dx = 0, dy = 0, dz = 0;
    if (v < nv) {
      dx = v % side - E;
      dy = (v / side) % side - E;
      dz = v / (side * side) - E;
      k = coverage(g, c, dx, dy, dz);
    }
    const int flag = k > 0;
    const unsigned bal = __ballot_sync(0xffffffffu, flag);
    const int rank = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    int pre = 0, tot = 0;
    for (int q = 0; q < nw; ++q) {
      if (q < w) pre += wsum[q];
      tot += wsum[q];
    }
    if (flag) {
      const int at = base_s + pre + rank;
      if (at < ptr[blockIdx.x + 1]) {
        off[at] = pack_off(dx, dy, dz);
        cnt[at] = (uint8_t)k;
      } else {
        atomicExch(err, 2);
      }
      if (dx == -E || dx == E || dy == -E || dy == E || dz == -E || dz == E) atomicExch(err, 3);
    }
    __syncthreads();
    if (threadIdx.x == 0) base_s += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (base_s != ptr[blockIdx.x + 1]) atomicExch(err, 2);
    alpha[blockIdx.x] = g.v_over_h3 / (double)sumcnt[blockIdx.x];
  }
}

// ---------------------------------------------------------------- voxelisation
template <class Q>
__device__ __forceinline__ void fixed_add(Q* p, long long v);
template <>
__device__ __forceinline__ void fixed_add<int32_t>(int32_t* p, long long v) {
  atomicAdd(reinterpret_cast<int*>(p), (int)v);
}
template <>
__device__ __forceinline__ void fixed_add<int64_t>(int64_t* p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

__device__ __forceinline__ int wrap(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// Fixed-point value of one stencil entry: floor(val + u) with u in [0, 1) drawn from a
// hash of the entry's index k and the component.  Its mean over u is val exactly, and the
// errors of different entries are independent.  Rounding to nearest would give every
// voxel of a loop that has the same coverage count (most of them) the same error, a
// coherent change of the loop's whole eigenstrain by up to half a quantum per voxel:
// 1.5e-8 relative for a <100> loop, 1.5e-5 eV of its 860 eV self term at 256^3.  A
// function of (k, comp) only, so a later removal subtracts the very same integer.
__device__ __forceinline__ long long fixed_of(double val, int k, int comp) {
  uint32_t h = (uint32_t)k * 6u + (uint32_t)comp;
  h ^= h >> 16;
  h *= 0x7feb352dU;
  h ^= h >> 15;
  h *= 0x846ca68bU;
  h ^= h >> 16;
  const double u = (double)(h >> 8) * (1.0 / 16777216.0);
  return __double2ll_rd(val + u);
}

// Adds sign * (count * alpha * eps*) of the class-c stencil of defect i placed at
// half-lattice position pos to the fixed-point field (quantum q, limit lim).
template <class Q>
__device__ void scatter_stencil(Q* __restrict__ eps, int3 n, size_t N, const DefGeo& g, const int* __restrict__ ptr,
                                const int* __restrict__ off, const uint8_t* __restrict__ cnt, const double* __restrict__ alpha,
                                int i, const int pos[3], int sign, double rq, double lim, int* err, int* dirty,
                                int slice = 0, int nslices = 1) {
  const int c = pos[0] & 1;
  const int bx = floor_div2(pos[0]), by = floor_div2(pos[1]), bz = floor_div2(pos[2]);
  const int s = ptr[2 * i + c], e = ptr[2 * i + c + 1];
  const double a = alpha[2 * i + c];
  for (int k = s + slice * blockDim.x + threadIdx.x; k < e; k += nslices * blockDim.x) {
    int dx, dy, dz;
    unpack_off(off[k], dx, dy, dz);
    const int zz = wrap(bz + dz, n.z);
    const size_t v = ((size_t)zz * n.y + wrap(by + dy, n.y)) * n.x + wrap(bx + dx, n.x);
    const double w = (double)cnt[k] * a;
    for (int comp = 0; comp < 6; ++comp) {
      const double val = w * g.e6[comp] * rq;
      if (fabs(val) > lim) atomicExch(err, 4);
      const long long iv = fixed_of(val, k, comp);
      if (iv) {
        fixed_add<Q>(eps + comp * N + v, sign * iv);
        if (dirty) dirty[comp * n.z + zz] = 1;  // same value from every writer
      }
    }
  }
}

// ---------------------------------------------------------------- energy lists
// The eight candidate positions of a defect in class c use the stencil of class
// cp = 1 - c shifted by s_j, s_j per axis in {-cp, 1 - cp} (bit 2 of j: x, bit 1: y,
// bit 0: z).  Their voxels are the 2x2x2 dilation of that stencil, and the site's own
// class-c stencil lies inside the same box.  For the energies each voxel u of the union
// is listed once with the site count and the eight counts cnt(u - s_j) (packed in a
// uint64), so sigma at u is read once for all nine positions.  One block per (defect,
// class c); the count box of both stencils lives in shared memory (side 2E + 1, E the
// scan half-width; class c' counts in the low byte, class c in the high byte), and
// lists come out in the box's linear order.
constexpr int kDilateMaxSide = 48;  // 2 * 48^3 bytes of shared memory; larger defects use the direct loops

__device__ __forceinline__ int dilate_prepare(const DefGeo& g, const int* __restrict__ ptr, const int* __restrict__ off,
                                              const uint8_t* __restrict__ cnt, int i, int cp, uint16_t* box) {
  const int E = g.extent, side = 2 * E + 1;
  const int nv = side * side * side;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) box[v] = 0;
  __syncthreads();
  for (int k = ptr[2 * i + cp] + threadIdx.x; k < ptr[2 * i + cp + 1]; k += blockDim.x) {
    int dx, dy, dz;
    unpack_off(off[k], dx, dy, dz);
    box[((dz + E) * side + (dy + E)) * side + (dx + E)] = cnt[k];
  }
  __syncthreads();
  const int c = 1 - cp;  // the site's own stencil, in the high byte (each voxel once)
  for (int k = ptr[2 * i + c] + threadIdx.x; k < ptr[2 * i + c + 1]; k += blockDim.x) {
    int dx, dy, dz;
    unpack_off(off[k], dx, dy, dz);
    uint16_t& b = box[((dz + E) * side + (dy + E)) * side + (dx + E)];
    b = (uint16_t)(b | ((unsigned)cnt[k] << 8));
  }
  __syncthreads();
  return nv;
}

__device__ __forceinline__ unsigned long long dilate_counts(const uint16_t* box, int E, int cp, int ux, int uy, int uz) {
  const int side = 2 * E + 1;
  unsigned long long cc = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int x = ux - (((j >> 2) & 1) - cp), y = uy - (((j >> 1) & 1) - cp), z = uz - ((j & 1) - cp);
    if (x >= -E && x <= E && y >= -E && y <= E && z >= -E && z <= E)
      cc |= (unsigned long long)(box[((z + E) * side + (y + E)) * side + (x + E)] & 255u) << (8 * j);
  }
  return cc;
}

__global__ void k_dilate_count(const DefGeo* __restrict__ G, const int* __restrict__ ptr, const int* __restrict__ off,
                               const uint8_t* __restrict__ cnt, int* __restrict__ ndil) {
  extern __shared__ uint16_t box[];
  __shared__ long long sh[32];
  const int i = blockIdx.x >> 1, c = blockIdx.x & 1, cp = 1 - c;
  const DefGeo g = G[i];
  const int E = g.extent, side = 2 * E + 1;
  if (side > kDilateMaxSide) {
    if (threadIdx.x == 0) ndil[blockIdx.x] = -1;
    return;
  }
  const int nv = dilate_prepare(g, ptr, off, cnt, i, cp, box);
  long long n = 0;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const int ux = v % side - E, uy = (v / side) % side - E, uz = v / (side * side) - E;
    n += (dilate_counts(box, E, cp, ux, uy, uz) != 0ull) || (box[v] >> 8) != 0;
  }
  n = block_sum_ll(n, sh);
  if (threadIdx.x == 0) ndil[blockIdx.x] = (int)n;
}

__global__ void k_dilate_fill(const DefGeo* __restrict__ G, const int* __restrict__ ptr, const int* __restrict__ off,
                              const uint8_t* __restrict__ cnt, DilatedLists dl, int* __restrict__ doff,
                              unsigned long long* __restrict__ dcnt, uint8_t* __restrict__ dscnt, int* __restrict__ err) {
  extern __shared__ uint16_t box[];
  __shared__ int wsum[32];
  const int i = blockIdx.x >> 1, c = blockIdx.x & 1, cp = 1 - c;
  const DefGeo g = G[i];
  const int E = g.extent, side = 2 * E + 1;
  if (side > kDilateMaxSide || dl.ptr[blockIdx.x] < 0) return;
  const int nv = dilate_prepare(g, ptr, off, cnt, i, cp, box);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int base = dl.ptr[blockIdx.x];
  const int end = dl.end[blockIdx.x];
  for (int v0 = 0; v0 < nv; v0 += blockDim.x) {
    const int v = v0 + threadIdx.x;
    int ux = 0, uy = 0, uz = 0;
    unsigned long long cc = 0;
    unsigned sc = 0;
    if (v < nv) {
      ux = v % side - E;
      uy = (v / side) % side - E;
      uz = v / (side * side) - E;
      cc = dilate_counts(box, E, cp, ux, uy, uz);
      sc = box[v] >> 8;
    }
    const bool any = cc != 0ull || sc != 0u;
    const unsigned bal = __ballot_sync(0xffffffffu, any);
    const int rank = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    int pre = 0, tot = 0;
    for (int q = 0; q < nw; ++q) {
      if (q < w) pre += wsum[q];
      tot += wsum[q];
    }
    if (any) {
      const int at = base + pre + rank;
      if (at < end) {
        doff[at] = pack_off(ux, uy, uz);
        dcnt[at] = cc;
        dscnt[at] = (uint8_t)sc;
      } else {
        atomicExch(err, 5);
      }
    }
    base += tot;
    __syncthreads();
  }
}

template <class Q>
__global__ void k_voxelise(Q* __restrict__ eps, int3 n, const okmc_defect* __restrict__ d, const DefGeo* __restrict__ G,
                           const int* __restrict__ ptr, const int* __restrict__ off, const uint8_t* __restrict__ cnt,
                           const double* __restrict__ alpha, double rq, double lim, int* err) {
  const int i = blockIdx.x;
  const size_t N = (size_t)n.x * n.y * n.z;
  const int pos[3] = {d[i].pos[0], d[i].pos[1], d[i].pos[2]};
  scatter_stencil<Q>(eps, n, N, G[i], ptr, off, cnt, alpha, i, pos, +1, rq, lim, err, nullptr);
}

// Blocks (move, slice): each slice of a move removes its share of the old stencil and
// adds its share of the new one (exact in fixed point, in any order).  Several slices
// per move spread the FP64 fixed-point conversions over several SMs.
constexpr int kMoveSlices = 16;
template <class Q>
__global__ void k_apply_moves(Q* __restrict__ eps, int3 n, const DefGeo* __restrict__ G, const int* __restrict__ ptr,
                              const int* __restrict__ off, const uint8_t* __restrict__ cnt, const double* __restrict__ alpha,
                              const Move* __restrict__ moves, const DevState* __restrict__ st, double rq, double lim, int* err,
                              int* dirty) {
  if ((int)blockIdx.x >= st->nmoves) return;
  const Move m = moves[blockIdx.x];
  const size_t N = (size_t)n.x * n.y * n.z;
  scatter_stencil<Q>(eps, n, N, G[m.i], ptr, off, cnt, alpha, m.i, m.old_pos, -1, rq, lim, err, dirty, blockIdx.y,
                     gridDim.y);
  scatter_stencil<Q>(eps, n, N, G[m.i], ptr, off, cnt, alpha, m.i, m.new_pos, +1, rq, lim, err, dirty, blockIdx.y,
                     gridDim.y);
}

// Moves recorded from a host-side position update.
__global__ void k_diff_positions(okmc_defect* __restrict__ d, const int* __restrict__ pos, int nd, Move* moves,
                                 DevState* st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  const int p0 = pos[3 * i], p1 = pos[3 * i + 1], p2 = pos[3 * i + 2];
  if (p0 != d[i].pos[0] || p1 != d[i].pos[1] || p2 != d[i].pos[2]) {
    const int k = atomicAdd(&st->nmoves, 1);
    Move m;
    m.i = i;
    m.old_pos[0] = d[i].pos[0];
    m.old_pos[1] = d[i].pos[1];
    m.old_pos[2] = d[i].pos[2];
    m.new_pos[0] = p0;
    m.new_pos[1] = p1;
    m.new_pos[2] = p2;
    moves[k] = m;
    d[i].pos[0] = p0;
    d[i].pos[1] = p1;
    d[i].pos[2] = p2;
  }
}

__global__ void k_gather_positions(const okmc_defect* __restrict__ d, int* __restrict__ pos, int nd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  pos[3 * i] = d[i].pos[0];
  pos[3 * i + 1] = d[i].pos[1];
  pos[3 * i + 2] = d[i].pos[2];
}

template <class Q, class T>
__global__ void k_fixed_to_real(const Q* __restrict__ eps, T* __restrict__ out, size_t total, double q) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x)
    out[k] = (T)((double)eps[k] * q);
}

// ---------------------------------------------------------------- self-term table
// Scalar count fields of up to six stencils (defect b.idx[f/2], class f%2), each
// placed with its base voxel at the origin.
template <class Q>
__global__ void k_wfields(Q* __restrict__ f, int3 n, const int* __restrict__ ptr, const int* __restrict__ off,
                          const uint8_t* __restrict__ cnt, WBatch b) {
  const int fi = blockIdx.x;
  if (fi >= 2 * b.nb) return;
  const size_t N = (size_t)n.x * n.y * n.z;
  const int i = b.idx[fi / 2], c = fi & 1;
  for (int k = ptr[2 * i + c] + threadIdx.x; k < ptr[2 * i + c + 1]; k += blockDim.x) {
    int dx, dy, dz;
    unpack_off(off[k], dx, dy, dz);
    const size_t v = ((size_t)wrap(dz, n.z) * n.y + wrap(dy, n.y)) * n.x + wrap(dx, n.x);
    fixed_add<Q>(f + fi * N + v, (long long)cnt[k]);
  }
}

// q(xi) = e : M(xi) : e with M = C Gamma C - C: for xi != 0, q = v . K^-1 v - tau : e with
// tau = C:e and v = tau m; at xi = 0, q = 0 (zero mean stress) or -tau : e (zero mean
// strain).  Averaged over the Nyquist sign as in the solve.
template <class T>
__device__ __forceinline__ T q_of(const T* tau, T te, T m0, T m1, T m2, T C11, T C12, T C44) {
  const T A = C11 - C12 - T(2) * C44, B = C12 + C44;
  const T k00 = C44 + (A + B) * m0 * m0, k11 = C44 + (A + B) * m1 * m1, k22 = C44 + (A + B) * m2 * m2;
  const T k01 = B * m0 * m1, k02 = B * m0 * m2, k12 = B * m1 * m2;
  const T i00 = k11 * k22 - k12 * k12, i01 = k02 * k12 - k01 * k22, i02 = k01 * k12 - k02 * k11;
  const T i11 = k00 * k22 - k02 * k02, i12 = k01 * k02 - k00 * k12, i22 = k00 * k11 - k01 * k01;
  const T det = k00 * i00 + k01 * i01 + k02 * i02;
  const T v0 = tau[0] * m0 + tau[5] * m1 + tau[4] * m2;
  const T v1 = tau[5] * m0 + tau[1] * m1 + tau[3] * m2;
  const T v2 = tau[4] * m0 + tau[3] * m1 + tau[2] * m2;
  const T vkv = v0 * (i00 * v0 + i01 * v1 + i02 * v2) + v1 * (i01 * v0 + i11 * v1 + i12 * v2) +
                v2 * (i02 * v0 + i12 * v1 + i22 * v2);
  return vkv / det - te;
}


// Frequency of half-spectrum index (kx, ky, kz) as a unit vector (signed frequencies,
// Nyquist index -N/2); false at xi = 0.
__device__ __forceinline__ bool unit_freq(const PassCfg& c, int kx, int ky, int kz, double& m0, double& m1, double& m2) {
  const int fx = kx < c.H ? kx : kx - c.nx;
  const int fy = ky < c.ny / 2 ? ky : ky - c.ny;
  const int fz = kz < c.nz / 2 ? kz : kz - c.nz;
  if (fx == 0 && fy == 0 && fz == 0) return false;
  const double qx = (double)fx / c.nx, qy = (double)fy / c.ny, qz = (double)fz / c.nz;
  const double rn = 1.0 / sqrt(qx * qx + qy * qy + qz * qz);
  m0 = qx * rn;
  m1 = qy * rn;
  m2 = qz * rn;
  return true;
}

// A value of Q_t rounded to the table precision.  FP32: rounded up or down at random
// (a hash of the table index), up with probability (v - lo)/(hi - lo), so that the
// stored value is v on average.  A loop's spectrum lies in a narrow cone about its
// normal, where Q_t hardly varies: rounded to nearest, all of those frequencies would
// carry the same rounding error, a coherent relative error of up to 3e-8 in the loop's
// self term (2e-5 eV for a 4 nm <100> loop); rounded at random, the errors are
// independent and average out over the cone.
template <class QT>
__device__ __forceinline__ QT table_value(double v, size_t idx);
template <>
__device__ __forceinline__ double table_value<double>(double v, size_t) { return v; }
template <>
__device__ __forceinline__ float table_value<float>(double v, size_t idx) {
  const float lo = __double2float_rd(v), hi = __double2float_ru(v);
  if (lo == hi) return lo;
  uint32_t h = (uint32_t)idx ^ (uint32_t)(idx >> 32) * 0x9e3779b9U;
  h ^= h >> 16;
  h *= 0x7feb352dU;
  h ^= h >> 15;
  h *= 0x846ca68bU;
  h ^= h >> 16;
  const double u = (double)(h >> 8) * (1.0 / 16777216.0);
  return u * ((double)hi - (double)lo) < v - (double)lo ? hi : lo;
}

// Q_t(xi) = E_t : M(xi) : E_t for each defect type present, [t][kz][p].  It is
// evaluated in FP64 whatever the field precision (a difference of two terms of
// similar size; an FP32 evaluation biases the self terms by ~2e-7 relative) and
// stored in QT (table_value).  A defect's q is s^2 Q_t with e = s E_t.
template <class QT>
__global__ void __launch_bounds__(256) k_qtable(QT* __restrict__ out, PassCfg c, QTypes qt) {
  const size_t P = (size_t)(c.H + 1) * c.ny;
  const size_t total = P * c.nz;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int kz = (int)(idx / P);
    const int p = (int)(idx % P);
    const int kx = p / c.ny, ky = p % c.ny;
    double m0, m1, m2;
    const bool nz0 = unit_freq(c, kx, ky, kz, m0, m1, m2);
    const bool nx_ = (kx == c.H), ny_ = (2 * ky == c.ny), nz_ = (2 * kz == c.nz);
    for (int t = 0; t < qt.nt; ++t) {
      const double* e = qt.e6[t];
      const double tr = e[0] + e[1] + e[2];
      double tau[6];
      for (int a = 0; a < 3; ++a) tau[a] = c.C12 * tr + (c.C11 - c.C12) * e[a];
      for (int a = 3; a < 6; ++a) tau[a] = 2.0 * c.C44 * e[a];
      const double te = tau[0] * e[0] + tau[1] * e[1] + tau[2] * e[2] + 2.0 * (tau[3] * e[3] + tau[4] * e[4] + tau[5] * e[5]);
      double v;
      if (!nz0) {
        v = (c.k0_mode == OKMC_MEAN_STRAIN_ZERO) ? -te : 0.0;
      } else {
        v = q_of<double>(tau, te, m0, m1, m2, c.C11, c.C12, c.C44);
        if (nx_ || ny_ || nz_)
          v = 0.5 * (v + q_of<double>(tau, te, nx_ ? -m0 : m0, ny_ ? -m1 : m1, nz_ ? -m2 : m2, c.C11, c.C12, c.C44));
      }
      out[(size_t)t * total + idx] = table_value<QT>(v, (size_t)t * total + idx);
    }
  }
}

// Per-thread accumulators of the self-term sums: compensated FP32 pairs for FP32
// spectra, plain FP64 for FP64 spectra.
template <class T> struct WAcc;
template <> struct WAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <> struct WAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};

// Sums over the half spectrum (weight 2 off the kx = 0 and kx = nx/2 planes) of
// Q_t(xi) |w0|^2, Q_t |w1|^2 and Q_t Re(conj(w1) w0 exp(i xi.d)) for the eight
// d in {-1, 0}^3, per defect of the batch; the products are formed in the
// spectrum precision.
template <class T, class QT>
__global__ void __launch_bounds__(256) k_selfterm_partial(const C2<T>* __restrict__ spec, PassCfg c, WBatch b,
                                                          const QT* __restrict__ qtab, const double2* __restrict__ phx,
                                                          const double2* __restrict__ phy, const double2* __restrict__ phz,
                                                          double* __restrict__ partial) {
  __shared__ double sh[32];
  const size_t P = (size_t)(c.H + 1) * c.ny;
  const size_t total = P * c.nz;
  WAcc<T> acc[3][10];
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int kz = (int)(idx / P);
    const int p = (int)(idx % P);
    const int kx = p / c.ny, ky = p % c.ny;
    const T wgt = (kx == 0 || kx == c.H) ? T(1) : T(2);
    // phase factors: bit 2 (x), 1 (y), 0 (z) clear means d = -1 on that axis, i.e. a
    // factor conj(e_axis)
    const double2 ex = phx[kx], ey = phy[ky], ez = phz[kz];
    const C2<T> ax{(T)ex.x, (T)-ex.y}, ay{(T)ey.x, (T)-ey.y}, az{(T)ez.x, (T)-ez.y};
    C2<T> ph[8];
    ph[7] = C2<T>{T(1), T(0)};
    ph[6] = az;
    ph[5] = ay;
    ph[4] = ay * az;
    ph[3] = ax;
    ph[2] = ax * az;
    ph[1] = ax * ay;
    ph[0] = ph[1] * az;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (d >= b.nb) break;
      const C2<T> w0 = spec[((size_t)(2 * d) * c.nz + kz) * P + p];
      const C2<T> w1 = spec[((size_t)(2 * d + 1) * c.nz + kz) * P + p];
      const T q = wgt * (T)qtab[(size_t)b.type[d] * total + idx];
      acc[d][0].add(q * (w0.x * w0.x + w0.y * w0.y));
      acc[d][1].add(q * (w1.x * w1.x + w1.y * w1.y));
      // conj(w1) * w0
      const T cr = w1.x * w0.x + w1.y * w0.y, ci = w1.x * w0.y - w1.y * w0.x;
      const T qr = q * cr, qi = q * ci;
#pragma unroll
      for (int s = 0; s < 8; ++s) acc[d][2 + s].add(qr * ph[s].x - qi * ph[s].y);
    }
  }
  for (int d = 0; d < 3; ++d)
    for (int k = 0; k < 10; ++k) {
      const double t = block_sum_d(acc[d][k].value(), sh);
      if (threadIdx.x == 0) partial[(size_t)blockIdx.x * 30 + d * 10 + k] = t;
    }
}

// W[i][c][0] = pref a_c^2 s^2 S_cc;  W[i][0][1+j] = pref a_0 a_1 s^2 X[d0(lambda_j)],
// d0 = (lambda - 1)/2 in {-1,0}^3;  W[i][1][1+j] = W[i][0][1+(7-j)] (the reverse jump).
__global__ void k_selfterm_final(const double* __restrict__ partial, int nblocks, WBatch b,
                                 const double* __restrict__ alpha, double pref, double* __restrict__ W) {
  const int d = threadIdx.x / 10, k = threadIdx.x % 10;
  __shared__ double S[30];
  if (threadIdx.x < 30) {
    double t = 0.0;
    for (int bl = 0; bl < nblocks; ++bl) t += partial[(size_t)bl * 30 + threadIdx.x];
    S[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x >= 30 || d >= b.nb || k) return;
  const int i = b.idx[d];
  const double a0 = alpha[2 * i], a1 = alpha[2 * i + 1];
  const double ps = pref * b.s2[d];
  double* w = W + (size_t)i * 18;
  w[0] = ps * a0 * a0 * S[d * 10 + 0];
  w[9] = ps * a1 * a1 * S[d * 10 + 1];
  // lambda_j components sx = +-1 -> d0 = 0 (sx = +1) or -1 (sx = -1); bit set means d = 0,
  // the same encoding as j (bit 2: sx > 0, bit 1: sy > 0, bit 0: sz > 0)
  for (int j = 0; j < 8; ++j) w[1 + j] = ps * a0 * a1 * S[d * 10 + 2 + j];
  for (int j = 0; j < 8; ++j) w[10 + j] = w[1 + (7 - j)];
}

// ---------------------------------------------------------------- energies
// E_i(Y) = -kappa h^3 alpha sum_v count(v - base(Y)) e_i : sigma(v) - W_i(c, lambda),
// for Y = X_i and the eight jumps.  Each product count * (e : sigma) is formed in the
// field precision and accumulated per thread as a compensated pair (TwoSum), the
// pairs are combined across the warp by compensated shuffles, and the per-warp
// results are added in FP64: the sums keep ~48 significant bits without FP64
// arithmetic in the inner loop.  Blocks visit defects largest stencil first.
struct CSum {
  float s, c;
};
__device__ __forceinline__ void csum_add(CSum& a, float x) {
  const float t = a.s + x;
  const float bp = t - a.s;
  a.c += (a.s - (t - bp)) + (x - bp);
  a.s = t;
}
__device__ __forceinline__ double csum_value(const CSum& a) { return (double)a.s + (double)a.c; }

static_assert(kEnergyWarpEntries == 4 * 32, "one pass of the unrolled loop (U = 4) of one warp");


template <class T>
struct EAcc;
template <>
struct EAcc<float> {
  CSum v;
  __device__ __forceinline__ void zero() { v = CSum{0.f, 0.f}; }
  __device__ __forceinline__ void add(float x) { csum_add(v, x); }
  // pairwise TwoSum of (s, c) pairs across the warp
  __device__ __forceinline__ void warp_reduce() {
    for (int o = 16; o; o >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, v.s, o), oc = __shfl_xor_sync(0xffffffffu, v.c, o);
      const float t = v.s + os, bp = t - v.s;
      const float err = (v.s - (t - bp)) + (os - bp);
      v.c = v.c + oc + err;
      v.s = t;
    }
  }
  __device__ __forceinline__ double value() const { return csum_value(v); }
};
template <>
struct EAcc<double> {
  double v;
  __device__ __forceinline__ void zero() { v = 0.0; }
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void warp_reduce() {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  __device__ __forceinline__ double value() const { return v; }
};

// The energies (and rates) of defect i, by a group of GS threads: the whole block
// (GS = kEnergyThreads) or one warp (GS = 32, for a defect whose energy list has at most
// kEnergyWarpEntries entries, one pass of the unrolled loop).  Thread gt of the group takes
// entries first + gt + m * GS.
template <class T, int GS>
__device__ __forceinline__ void energies_item(const T* __restrict__ sig, int3 n, const okmc_defect* __restrict__ d,
                                              const DefGeo* __restrict__ G, const int* __restrict__ ptr,
                                              const int* __restrict__ off, const uint8_t* __restrict__ cnt,
                                              const double* __restrict__ alpha, const double* __restrict__ W, double pref,
                                              int want_cand, int i, double* __restrict__ E, double* __restrict__ Ec,
                                              const RateArgs& ra, const DilatedLists& dl) {
  // per-warp partial sums: FP32 (sum, compensation) pairs for FP32 fields, converted to
  // FP64 only in the epilogue warp (each conversion of a warp costs a whole FP64 issue
  // slot, even with one lane active); FP64 sums for FP64 fields
  static_assert(GS == 32 || GS == kEnergyThreads, "a warp or the whole block");
  __shared__ T part[kEnergyThreads / 32][9];
  __shared__ T partc[kEnergyThreads / 32][9];
  const size_t N = (size_t)n.x * n.y * n.z;
  const int gt = GS == 32 ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool ep = GS == 32 || threadIdx.x < 32;  // the warp that runs the epilogue
  const okmc_defect r = d[i];
  const DefGeo g = G[i];
  const int c = r.pos[0] & 1, cp = 1 - c;
  // the epilogue's inputs, loaded now so that they arrive while the sums run
  double al = 0.0, wv = 0.0, es = 0.0;
  if (ep && lane < 9) {
    al = alpha[2 * i + (lane == 0 ? c : cp)];
    wv = W[(size_t)i * 18 + c * 9 + lane];
    es = G[i].escale;
  }
  // the weights e_i (off-diagonals twice) in units of the defect's scale, whose FP64
  // value multiplies the sums at the end: every weight is 0, +-1 or +-2, exact in FP32,
  // whereas e itself rounded to FP32 (1/(2 sqrt 3) for a 1/2<111> loop: -1.8e-8
  // relative) would bias every sum, self part included, by that ratio
  T ew[6];
  for (int a = 0; a < 6; ++a) ew[a] = T(g.ew[a]);
  // components with zero weight (a <100> loop needs sigma_xx only, a dilatation the
  // trace) are not gathered; adding their zero products would not change any sum
  bool use[6];
  for (int a = 0; a < 6; ++a) use[a] = ew[a] != T(0);
  const int bx = floor_div2(r.pos[0]), by = floor_div2(r.pos[1]), bz = floor_div2(r.pos[2]);
  EAcc<T> acc[9];
  for (int j = 0; j < 9; ++j) acc[j].zero();
  // Each thread takes the entries k = first + tid + m * blockDim in order; U of them at
  // a time, with every load of the group issued before the first use, so that U
  // gathers are in flight per thread (the accumulation order is that of the plain loop).
  constexpr int U = 4;
  if (want_cand && dl.ptr && dl.ptr[2 * i + c] >= 0) {
    // the energy list: each voxel of the site and candidate stencils once, nine counts
    const int k_end = dl.end[2 * i + c];
    for (int k0 = dl.ptr[2 * i + c] + gt; k0 < k_end; k0 += U * GS) {
      T sv[U][6];
      unsigned long long cc[U];
      unsigned sc[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = k0 + u * GS;
        cc[u] = 0ull;
        sc[u] = 0u;
        if (k < k_end) {
          int ux, uy, uz;
          unpack_off(dl.off[k], ux, uy, uz);
          cc[u] = dl.cnt[k];
          sc[u] = dl.scnt[k];
          const size_t v = ((size_t)wrap(bz + uz, n.z) * n.y + wrap(by + uy, n.y)) * n.x + wrap(bx + ux, n.x);
#pragma unroll
          for (int a = 0; a < 6; ++a) sv[u][a] = use[a] ? __ldg(sig + a * N + v) : T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (k0 + u * GS >= k_end) break;
        T dot = T(0);
#pragma unroll
        for (int a = 0; a < 6; ++a) dot += ew[a] * sv[u][a];
        if (sc[u]) acc[0].add(T(sc[u]) * dot);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[1 + j].add(T((unsigned)(cc[u] >> (8 * j)) & 255u) * dot);
      }
    }
  } else {
    {  // the site stencil
      const int k_end = ptr[2 * i + c + 1];
      for (int k0 = ptr[2 * i + c] + gt; k0 < k_end; k0 += U * GS) {
        T sv[U][6], w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int k = k0 + u * GS;
          w[u] = T(0);
          if (k < k_end) {
            int dx, dy, dz;
            unpack_off(off[k], dx, dy, dz);
            w[u] = T(cnt[k]);
            const size_t v = ((size_t)wrap(bz + dz, n.z) * n.y + wrap(by + dy, n.y)) * n.x + wrap(bx + dx, n.x);
#pragma unroll
            for (int a = 0; a < 6; ++a) sv[u][a] = use[a] ? __ldg(sig + a * N + v) : T(0);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (k0 + u * GS >= k_end) break;
          T dot = T(0);
#pragma unroll
          for (int a = 0; a < 6; ++a) dot += ew[a] * sv[u][a];
          acc[0].add(w[u] * dot);
        }
      }
    }
    if (want_cand) {
      // candidate j sits at base(X + lambda_j) = base(X) + d_j, d_j in {-1,0}^3 (c = 0)
      // or {0,1}^3 (c = 1); per axis the shift is (s + 1)/2 - (1 - c) with s = +-1
      for (int k = ptr[2 * i + cp] + gt; k < ptr[2 * i + cp + 1]; k += GS) {
        int dx, dy, dz;
        unpack_off(off[k], dx, dy, dz);
        const T w = T(cnt[k]);
        const int x0 = wrap(bx + dx - cp, n.x), x1 = wrap(bx + dx + 1 - cp, n.x);
        const int y0 = wrap(by + dy - cp, n.y), y1 = wrap(by + dy + 1 - cp, n.y);
        const int z0 = wrap(bz + dz - cp, n.z), z1 = wrap(bz + dz + 1 - cp, n.z);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const size_t v = ((size_t)((j & 1) ? z1 : z0) * n.y + ((j & 2) ? y1 : y0)) * n.x + ((j & 4) ? x1 : x0);
          T dot = T(0);
#pragma unroll
          for (int a = 0; a < 6; ++a) dot += ew[a] * (use[a] ? __ldg(sig + a * N + v) : T(0));
          acc[1 + j].add(w * dot);
        }
      }
    }
  }
  // warp reduction of the accumulators (compensated pairs stay FP32), FP64 across warps
  const int wid = threadIdx.x >> 5;
  double tot = 0.0;
  if constexpr (GS == 32) {
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      acc[j].warp_reduce();
      if (lane == j) tot = acc[j].value();
    }
  } else {
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      acc[j].warp_reduce();
      if (lane == 0) {
        if constexpr (sizeof(T) == 4) {
          part[wid][j] = acc[j].v.s;
          partc[wid][j] = acc[j].v.c;
        } else {
          part[wid][j] = acc[j].v;
          partc[wid][j] = T(0);
        }
      }
    }
    __syncthreads();
    // epilogue on warp 0, one lane per position (lane 0: the site, lane 1 + j: jump j),
    // so the FP64 work (sums, energies, Boltzmann factors) runs side by side
    if (threadIdx.x >= 32) return;
    if (lane < 9)
      for (int w2 = 0; w2 < GS / 32; ++w2) tot += (double)part[w2][lane] + (double)partc[w2][lane];
  }
  double ej = 0.0;
  if (lane < 9) ej = pref * es * al * tot - wv;
  const double e0 = __shfl_sync(0xffffffffu, ej, 0);
  if (lane == 0) E[i] = e0;
  if (!want_cand) return;
  if (lane >= 1 && lane < 9) Ec[(size_t)i * 8 + lane - 1] = ej;
  if (!ra.rates) return;
  // biased jump frequencies nu_j = (nu0/z) exp(-(E_m + (E_j - E_0)/2)/kT) of the
  // allowed jumps (Eqs. biased_forward/backward_boltzmann, prefactor 1/z)
  double nu = 0.0;
  int neg = 0;
  if (lane >= 1 && lane < 9) {
    const int j = lane - 1;
    if (g.allowed >> j & 1) {
      const double barrier = r.Em_eV + 0.5 * (ej - e0);
      neg = barrier < 0.0;
      nu = (ra.nu0 / g.z) * exp(-barrier * ra.rkT);
    }
    ra.rates[(size_t)i * 8 + j] = nu;
  }
  double sum = 0.0;  // in jump order, as the frequency line walks them
  for (int j = 0; j < 8; ++j) sum += __shfl_sync(0xffffffffu, nu, 1 + j);
  neg = __reduce_add_sync(0xffffffffu, neg);
  if (lane == 0) {
    ra.rsum[i] = sum;
    if (neg) atomicAdd(reinterpret_cast<unsigned long long*>(ra.negb), (unsigned long long)neg);
  }
}

// Blocks 0 .. nbig - 1 take the defects order[0 .. nbig - 1] (the large lists, largest
// first) one per block; each later block takes the next kEnergyThreads / 32 defects of
// the order, one per warp.
template <class T>
__global__ void __launch_bounds__(kEnergyThreads, sizeof(T) == 4 ? 4 : 2) k_energies(const T* __restrict__ sig, int3 n, const okmc_defect* __restrict__ d,
                                                             const DefGeo* __restrict__ G, const int* __restrict__ ptr,
                                                             const int* __restrict__ off, const uint8_t* __restrict__ cnt,
                                                             const double* __restrict__ alpha, const double* __restrict__ W,
                                                             double pref, int want_cand, const int* __restrict__ order,
                                                             double* __restrict__ E, double* __restrict__ Ec, RateArgs ra,
                                                             DilatedLists dl, int nd, int nbig) {
  if ((int)blockIdx.x < nbig) {
    energies_item<T, kEnergyThreads>(sig, n, d, G, ptr, off, cnt, alpha, W, pref, want_cand, order[blockIdx.x], E, Ec, ra, dl);
  } else {
    const int k = nbig + ((int)blockIdx.x - nbig) * (kEnergyThreads / 32) + (int)(threadIdx.x >> 5);
    if (k < nd) energies_item<T, 32>(sig, n, d, G, ptr, off, cnt, alpha, W, pref, want_cand, order[k], E, Ec, ra, dl);
  }
}

// ---------------------------------------------------------------- energies by chunks
// Chunk slot w of the energy lists, by one warp: the entries of one pass of the unrolled
// loop (each lane U of them, all loads issued before the first use), the nine sums
// accumulated per lane as in energies_item, combined across the warp, and stored as FP64
// (site sum, then jump j).  A slot beyond the current class's list stores nothing.
template <class T>
__device__ __forceinline__ void energy_chunk(const T* __restrict__ sig, int3 n, const okmc_defect* __restrict__ d,
                                             const DefGeo* __restrict__ G, const DilatedLists& dl, const ChunkArgs& ca,
                                             int w) {
  constexpr int U = kEnergyWarpEntries / 32;
  const int lane = threadIdx.x & 31;
  const int i = ca.cdef[w];
  const int k = w - ca.c0[i];
  int pos[3];
  for (int a = 0; a < 3; ++a) pos[a] = d[i].pos[a];
  const int c = pos[0] & 1;
  const int first = dl.ptr[2 * i + c] + k * kEnergyWarpEntries;
  const int k_end = min(first + kEnergyWarpEntries, dl.end[2 * i + c]);
  if (first >= k_end) return;
  const size_t N = (size_t)n.x * n.y * n.z;
  T ew[6];
  bool use[6];
  for (int a = 0; a < 6; ++a) {
    ew[a] = T(G[i].ew[a]);
    use[a] = ew[a] != T(0);
  }
  const int bx = floor_div2(pos[0]), by = floor_div2(pos[1]), bz = floor_div2(pos[2]);
  EAcc<T> acc[9];
  for (int j = 0; j < 9; ++j) acc[j].zero();
  T sv[U][6];
  unsigned long long cc[U];
  unsigned sc[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int kk = first + lane + 32 * u;
    cc[u] = 0ull;
    sc[u] = 0u;
    if (kk < k_end) {
      int ux, uy, uz;
      unpack_off(dl.off[kk], ux, uy, uz);
      cc[u] = dl.cnt[kk];
      sc[u] = dl.scnt[kk];
      const size_t v = ((size_t)wrap(bz + uz, n.z) * n.y + wrap(by + uy, n.y)) * n.x + wrap(bx + ux, n.x);
#pragma unroll
      for (int a = 0; a < 6; ++a) sv[u][a] = use[a] ? __ldg(sig + a * N + v) : T(0);
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (first + lane + 32 * u >= k_end) break;
    T dot = T(0);
#pragma unroll
    for (int a = 0; a < 6; ++a) dot += ew[a] * sv[u][a];
    if (sc[u]) acc[0].add(T(sc[u]) * dot);
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[1 + j].add(T((unsigned)(cc[u] >> (8 * j)) & 255u) * dot);
  }
  // lane j keeps sum j (FP32 moves), then one conversion per warp
  EAcc<T> mine;
  mine.zero();
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    acc[j].warp_reduce();
    if (lane == j) mine = acc[j];
  }
  if (lane < 9) ca.part[(size_t)w * 9 + lane] = mine.value();
}

// Defects 3q, 3q + 1, 3q + 2 by one warp, nine lanes each (lane 9g + j: defect 3q + g,
// position j: the site, then jump j - 1): the chunk sums in slot order, the energies,
// and, with ra.rates set, the biased jump frequencies and their sum, as in energies_item.
__device__ __forceinline__ void energy_finish(const okmc_defect* __restrict__ d, const DefGeo* __restrict__ G,
                                              const DilatedLists& dl, const ChunkArgs& ca,
                                              const double* __restrict__ alpha, const double* __restrict__ W,
                                              double pref, int nd, int q, double* __restrict__ E,
                                              double* __restrict__ Ec, const RateArgs& ra) {
  const int lane = threadIdx.x & 31, grp = lane / 9, j = lane - 9 * grp;
  const int i = 3 * q + grp;
  const bool act = grp < 3 && i < nd;
  double ej = 0.0, Em = 0.0, z = 1.0;
  unsigned allowed = 0u;
  if (act) {
    // every load that does not depend on the site class first (both classes' values),
    // then the class's chunk sums (every defect has at least one chunk)
    const int p0 = d[i].pos[0];
    Em = d[i].Em_eV;
    const int s0 = ca.c0[i];
    const int b0 = dl.ptr[2 * i], b1 = dl.ptr[2 * i + 1], e0_ = dl.end[2 * i], e1_ = dl.end[2 * i + 1];
    const double a0 = alpha[2 * i], a1 = alpha[2 * i + 1];
    const double w0 = W[(size_t)i * 18 + j], w1 = W[(size_t)i * 18 + 9 + j];
    const double es = G[i].escale;
    allowed = G[i].allowed;
    z = G[i].z;
    // every energy list holds at least the voxels of the site stencil, so every defect
    // owns at least one chunk slot and uses at least one
    const double* P = ca.part + (size_t)s0 * 9 + j;
    double tot = P[0];
    const int c = p0 & 1;
    const int nch = ((c ? e1_ - b1 : e0_ - b0) + kEnergyWarpEntries - 1) / kEnergyWarpEntries;
    for (int k = 1; k < nch; ++k) tot += P[(size_t)k * 9];
    const double al = (j == 0) == (c == 0) ? a0 : a1;  // alpha of the site's class, or of the other class for a jump
    ej = pref * es * al * tot - (c ? w1 : w0);
  }
  const double e0 = __shfl_sync(0xffffffffu, ej, (9 * grp) & 31);
  if (act && j == 0) E[i] = e0;
  if (act && j >= 1) Ec[(size_t)i * 8 + j - 1] = ej;
  if (!ra.rates) return;
  // biased jump frequencies nu_j = (nu0/z) exp(-(E_m + (E_j - E_0)/2)/kT) of the
  // allowed jumps (Eqs. biased_forward/backward_boltzmann, prefactor 1/z)
  double nu = 0.0;
  int neg = 0;
  if (act && j >= 1) {
    if (allowed >> (j - 1) & 1) {
      const double barrier = Em + 0.5 * (ej - e0);
      neg = barrier < 0.0;
      nu = (ra.nu0 / z) * exp(-barrier * ra.rkT);
    }
    ra.rates[(size_t)i * 8 + j - 1] = nu;
  }
  double sum = 0.0;  // in jump order, as the frequency line walks them
  for (int jj = 0; jj < 8; ++jj) sum += __shfl_sync(0xffffffffu, nu, (9 * grp + 1 + jj) & 31);
  neg = __reduce_add_sync(0xffffffffu, neg);
  if (act && j == 0) ra.rsum[i] = sum;
  if (lane == 0 && neg) atomicAdd(reinterpret_cast<unsigned long long*>(ra.negb), (unsigned long long)neg);
}

template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 3) k_energy_chunks(const T* __restrict__ sig, int3 n, const okmc_defect* __restrict__ d,
                                                       const DefGeo* __restrict__ G, DilatedLists dl, ChunkArgs ca) {
  const int w = (int)blockIdx.x * 8 + (int)(threadIdx.x >> 5);
  if (w < ca.nchunk) energy_chunk<T>(sig, n, d, G, dl, ca, w);
}

__global__ void __launch_bounds__(64) k_energy_finish(const okmc_defect* __restrict__ d, const DefGeo* __restrict__ G,
                                                      DilatedLists dl, ChunkArgs ca, const double* __restrict__ alpha,
                                                      const double* __restrict__ W, double pref, int nd,
                                                      double* __restrict__ E, double* __restrict__ Ec, RateArgs ra) {
  const int q = (int)blockIdx.x * 2 + (int)(threadIdx.x >> 5);
  if (3 * q < nd) energy_finish(d, G, dl, ca, alpha, W, pref, nd, q, E, Ec, ra);
}

// ---------------------------------------------------------------- events
__device__ __forceinline__ void new_position(const int p[3], int j, int3 n, int q[3]) {
  const int L[3] = {2 * n.x, 2 * n.y, 2 * n.z};
  for (int a = 0; a < 3; ++a) {
    int v = p[a] + jump_comp(j, a);
    if (v < 0) v += L[a];
    if (v >= L[a]) v -= L[a];
    q[a] = v;
  }
}

// Residence-time event: every allowed jump of every defect on one frequency line
// (i-major, j-minor, rates from the energies kernel), selection of the first entry
// whose running sum reaches u1 * R_tot (u1 in (0,1], Eq. selection_jump), clock
// advance -ln(u2)/R_tot.  One block: per-thread sums over a contiguous chunk of
// defects, a block scan, then the chunk that holds the target is walked.
constexpr int kEventThreads = 1024;
__device__ __forceinline__ void residence_item(okmc_defect* __restrict__ d, int nd, const double* __restrict__ rates,
                                               const double* __restrict__ rsum, int3 n, uint32_t key0, uint32_t key1,
                                               Move* __restrict__ moves, DevState* __restrict__ st) {
  __shared__ double wsum[kEventThreads / 32];
  __shared__ int sel_t, last_t;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int per = (nd + blockDim.x - 1) / blockDim.x;
  const int i0 = min(nd, t * per), i1 = min(nd, i0 + per);
  double s = 0.0;
  for (int i = i0; i < i1; ++i) s += rsum[i];
  // inclusive scan of the chunk sums: within each warp by shuffles, then over the
  // warp totals (fixed order, so the line is the same on every run)
  double v = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  double ex = __shfl_up_sync(0xffffffffu, v, 1);
  if (lane == 0) ex = 0.0;
  if (lane == 31) wsum[w] = v;
  if (t == 0) {
    sel_t = 0x7fffffff;
    last_t = -1;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    double x = lane < nw ? wsum[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane < nw) wsum[lane] = x;
  }
  __syncthreads();
  const double base = w > 0 ? wsum[w - 1] : 0.0;
  const double incl = base + v, excl = base + ex;
  const double R = wsum[(blockDim.x >> 5) - 1];
  const long long step = st->step;
  const uint32_t ctr[4] = {(uint32_t)step, (uint32_t)(step >> 32), 0xFFFFFFFFu, 0u};
  uint32_t x[4];
  philox4x32_10(ctr, key0, key1, x);
  const double u1 = u53(x[0], x[1]), u2 = u53(x[2], x[3]);
  const double target = u1 * R;
  // the first chunk whose running sum reaches the target (else the last nonzero one)
  const unsigned hit = __ballot_sync(0xffffffffu, s > 0.0 && incl >= target);
  const unsigned nz = __ballot_sync(0xffffffffu, s > 0.0);
  if (lane == 0) {
    if (hit) atomicMin(&sel_t, (w << 5) + __ffs(hit) - 1);
    if (nz) atomicMax(&last_t, (w << 5) + 31 - __clz(nz));
  }
  __syncthreads();
  const int pick_t = sel_t != 0x7fffffff ? sel_t : last_t;
  if (t != pick_t) {
    if (t == 0 && pick_t < 0) {  // no positive rate anywhere
      st->err = 5;
      st->nmoves = 0;
    }
    return;
  }
  double run = excl;
  int pi = -1, pj = -1, li = -1, lj = -1;
  for (int i = i0; i < i1 && pi < 0; ++i) {
    for (int j = 0; j < 8; ++j) {
      const double r = rates[(size_t)i * 8 + j];
      if (r <= 0.0) continue;
      li = i;
      lj = j;
      run += r;
      if (run >= target) {
        pi = i;
        pj = j;
        break;
      }
    }
  }
  if (pi < 0) {
    pi = li;
    pj = lj;
  }
  if (pi < 0 || !(R > 0.0)) {
    st->err = 5;
    st->nmoves = 0;
    return;
  }
  Move m;
  m.i = pi;
  for (int a = 0; a < 3; ++a) m.old_pos[a] = d[pi].pos[a];
  new_position(m.old_pos, pj, n, m.new_pos);
  for (int a = 0; a < 3; ++a) d[pi].pos[a] = m.new_pos[a];
  moves[0] = m;
  st->nmoves = 1;
  st->dt_last = -log(u2) / R;
  st->clock += st->dt_last;
  st->events += 1;
  st->step = step + 1;
}

__global__ void __launch_bounds__(kEventThreads) k_residence(okmc_defect* __restrict__ d, int nd,
                                                             const double* __restrict__ rates,
                                                             const double* __restrict__ rsum, int3 n, uint32_t key0,
                                                             uint32_t key1, Move* __restrict__ moves,
                                                             DevState* __restrict__ st) {
  residence_item(d, nd, rates, rsum, n, key0, key1, moves, st);
}

// Fixed time step (Algorithm 1): delta t = 1/max nominal nu over mobile defects;
// defect i fires when its Poisson count is > 0 (u_p > exp(-nu_i delta t)) and then
// selects a jump on its own biased frequency line with u_s.  One block.
__device__ __forceinline__ void fixed_dt_item(okmc_defect* __restrict__ d, const DefGeo* __restrict__ G, int nd,
                                              const double* __restrict__ rates, double nu0, double kT, int3 n, uint32_t key0,
                                              uint32_t key1, Move* __restrict__ moves, DevState* __restrict__ st) {
  __shared__ double red[32];
  __shared__ int cnt_s;
  const int t = threadIdx.x;
  double mx = 0.0;
  for (int i = t; i < nd; i += blockDim.x)
    if (G[i].z > 0) mx = fmax(mx, nu0 * exp(-d[i].Em_eV / kT));
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((t & 31) == 0) red[t >> 5] = mx;
  if (t == 0) cnt_s = 0;
  __syncthreads();
  double vmax = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) vmax = fmax(vmax, red[w]);
  const double dt = 1.0 / vmax;
  const long long step = st->step;
  for (int i = t; i < nd; i += blockDim.x) {
    const DefGeo g = G[i];
    if (g.z == 0) continue;
    const uint32_t ctr[4] = {(uint32_t)step, (uint32_t)(step >> 32), (uint32_t)i, 1u};
    uint32_t x[4];
    philox4x32_10(ctr, key0, key1, x);
    const double up = u53(x[0], x[1]), us = u53(x[2], x[3]);
    const double mu = nu0 * exp(-d[i].Em_eV / kT) * dt;
    if (up <= exp(-mu)) continue;
    double r[8], tot = 0.0;
    for (int j = 0; j < 8; ++j) {
      r[j] = rates[(size_t)i * 8 + j];
      tot += r[j];
    }
    const double target = us * tot;
    double run = 0.0;
    int pick = -1, last = -1;
    for (int j = 0; j < 8; ++j) {
      if (r[j] <= 0.0) continue;
      last = j;
      run += r[j];
      if (run >= target) {
        pick = j;
        break;
      }
    }
    if (pick < 0) pick = last;
    Move m;
    m.i = i;
    for (int a = 0; a < 3; ++a) m.old_pos[a] = d[i].pos[a];
    new_position(m.old_pos, pick, n, m.new_pos);
    const int k = atomicAdd(&cnt_s, 1);
    moves[k] = m;
  }
  __syncthreads();
  // apply all moves after every decision was taken from the start-of-step energies
  for (int k = t; k < cnt_s; k += blockDim.x) {
    const Move m = moves[k];
    for (int a = 0; a < 3; ++a) d[m.i].pos[a] = m.new_pos[a];
  }
  if (t == 0) {
    st->nmoves = cnt_s;
    st->dt_fixed = dt;
    st->dt_last = dt;
    st->clock += dt;
    st->events += cnt_s;
    st->step = step + 1;
  }
}

__global__ void __launch_bounds__(kEventThreads) k_fixed_dt(okmc_defect* __restrict__ d, const DefGeo* __restrict__ G, int nd,
                                                            const double* __restrict__ rates, double nu0, double kT,
                                                            int3 n, uint32_t key0, uint32_t key1,
                                                            Move* __restrict__ moves, DevState* __restrict__ st) {
  fixed_dt_item(d, G, nd, rates, nu0, kT, n, key0, key1, moves, st);
}

// ---------------------------------------------------------------- batched ensemble kernels
// One block per replica: its residence-time event or fixed-time step (Algorithm 1).
// The two passes of the chunked energies over work lists of (replica, chunk slot) and
// (replica, warp of three defects) items, one item per warp, persistent.
__global__ void __launch_bounds__(256, 4) k_energy_chunks_batch(const BatchRep* __restrict__ reps,
                                                             const int2* __restrict__ items, int nitems) {
  for (int it = (int)blockIdx.x * 8 + (int)(threadIdx.x >> 5); it < nitems; it += (int)gridDim.x * 8) {
    const int2 w = items[it];
    const BatchRep& r = reps[w.x];
    energy_chunk<float>(r.sig, r.n, r.def, r.geo, r.dl, r.ca, w.y);
  }
}
__global__ void __launch_bounds__(256) k_energy_finish_batch(const BatchRep* __restrict__ reps,
                                                             const int2* __restrict__ items, int nitems) {
  for (int it = (int)blockIdx.x * 8 + (int)(threadIdx.x >> 5); it < nitems; it += (int)gridDim.x * 8) {
    const int2 w = items[it];
    const BatchRep& r = reps[w.x];
    energy_finish(r.def, r.geo, r.dl, r.ca, r.alpha, r.W, r.pref, r.nd, w.y, r.E, r.Ec, r.ra);
  }
}

__global__ void __launch_bounds__(kEventThreads) k_event_batch(const BatchRep* __restrict__ reps) {
  const BatchRep& r = reps[blockIdx.x];
  if (r.mode == OKMC_RESIDENCE)
    residence_item(r.def, r.nd, r.ra.rates, r.ra.rsum, r.n, r.key0, r.key1, r.moves, r.state);
  else
    fixed_dt_item(r.def, r.geo, r.nd, r.ra.rates, r.nu0, r.kT, r.n, r.key0, r.key1, r.moves, r.state);
}

// Blocks (replica, slice): slice s of every move of the replica (old stencil out, new in;
// exact in fixed point, in any order), kMoveSlices slices per replica.
__global__ void __launch_bounds__(256) k_moves_batch(const BatchRep* __restrict__ reps) {
  const BatchRep& r = reps[blockIdx.x];
  const size_t N = (size_t)r.n.x * r.n.y * r.n.z;
  const int nm = r.state->nmoves;
  int32_t* eps = const_cast<int32_t*>(r.eps);
  for (int k = 0; k < nm; ++k) {
    const Move m = r.moves[k];
    scatter_stencil<int32_t>(eps, r.n, N, r.geo[m.i], r.ptr, r.off, r.cnt, r.alpha, m.i, m.old_pos, -1, r.rq, r.lim, r.err,
                             r.cfg.dirty, blockIdx.y, gridDim.y);
    scatter_stencil<int32_t>(eps, r.n, N, r.geo[m.i], r.ptr, r.off, r.cnt, r.alpha, m.i, m.new_pos, +1, r.rq, r.lim, r.err,
                             r.cfg.dirty, blockIdx.y, gridDim.y);
  }
}

cudaError_t launch_energy_chunks_batch(const BatchRep* reps, const int2* items, int nitems, int grid, cudaStream_t st) {
  if (nitems == 0) return cudaSuccess;
  k_energy_chunks_batch<<<grid, 256, 0, st>>>(reps, items, nitems);
  return cudaGetLastError();
}
cudaError_t launch_energy_finish_batch(const BatchRep* reps, const int2* items, int nitems, int grid, cudaStream_t st) {
  if (nitems == 0) return cudaSuccess;
  k_energy_finish_batch<<<grid, 256, 0, st>>>(reps, items, nitems);
  return cudaGetLastError();
}
cudaError_t launch_event_batch(const BatchRep* reps, int nrep, cudaStream_t st) {
  k_event_batch<<<nrep, kEventThreads, 0, st>>>(reps);
  return cudaGetLastError();
}
cudaError_t launch_moves_batch(const BatchRep* reps, int nrep, cudaStream_t st) {
  k_moves_batch<<<dim3(nrep, kMoveSlices), 256, 0, st>>>(reps);
  return cudaGetLastError();
}
// Blocks of the batched chunked-energies kernel resident on the device at once (its
// persistent grid; one work item per warp).
int energies_batch_grid() {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_energy_chunks_batch, 256, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    return 152 * 8;
  }
  return sms * (per > 0 ? per : 1);
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_defect_setup(const okmc_defect* d, DefGeo* G, int nd, double h, cudaStream_t st) {
  k_defect_setup<<<(nd + 127) / 128, 128, 0, st>>>(d, G, nd, h);
  return cudaGetLastError();
}
cudaError_t launch_stencil_count(const DefGeo* G, int nd, int* nnz, long long* sumcnt, cudaStream_t st) {
  k_stencil_count<<<2 * nd, 256, 0, st>>>(G, nnz, sumcnt);
  return cudaGetLastError();
}
cudaError_t launch_dilate_count(const DefGeo* G, int nd, const int* ptr, const int* off, const uint8_t* cnt, int* ndil,
                                cudaStream_t st) {
  const size_t smem = sizeof(uint16_t) * kDilateMaxSide * kDilateMaxSide * kDilateMaxSide;
  cudaError_t e = cudaFuncSetAttribute(k_dilate_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_dilate_count<<<2 * nd, 256, smem, st>>>(G, ptr, off, cnt, ndil);
  return cudaGetLastError();
}
cudaError_t launch_dilate_fill(const DefGeo* G, int nd, const int* ptr, const int* off, const uint8_t* cnt,
                               const DilatedLists& dl, int* err, cudaStream_t st) {
  const size_t smem = sizeof(uint16_t) * kDilateMaxSide * kDilateMaxSide * kDilateMaxSide;
  cudaError_t e = cudaFuncSetAttribute(k_dilate_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_dilate_fill<<<2 * nd, 256, smem, st>>>(G, ptr, off, cnt, dl, const_cast<int*>(dl.off),
                                           const_cast<unsigned long long*>(dl.cnt), const_cast<uint8_t*>(dl.scnt), err);
  return cudaGetLastError();
}
cudaError_t launch_stencil_fill(const DefGeo* G, int nd, const int* ptr, const long long* sumcnt, int* off, uint8_t* cnt,
                                double* alpha, int* err, cudaStream_t st) {
  k_stencil_fill<<<2 * nd, 256, 0, st>>>(G, ptr, sumcnt, off, cnt, alpha, err);
  return cudaGetLastError();
}
template <class Q>
cudaError_t launch_voxelise(Q* eps, int3 n, const okmc_defect* d, const DefGeo* G, int nd, const int* ptr, const int* off,
                            const uint8_t* cnt, const double* alpha, double rq, double lim, int* err, cudaStream_t st) {
  if (nd == 0) return cudaSuccess;
  k_voxelise<Q><<<nd, 256, 0, st>>>(eps, n, d, G, ptr, off, cnt, alpha, rq, lim, err);
  return cudaGetLastError();
}
template <class Q>
cudaError_t launch_apply_moves(Q* eps, int3 n, const DefGeo* G, int maxmoves, const int* ptr, const int* off,
                               const uint8_t* cnt, const double* alpha, const Move* moves, const DevState* stt, double rq,
                               double lim, int* err, int* dirty, cudaStream_t st) {
  if (maxmoves == 0) return cudaSuccess;
  k_apply_moves<Q><<<dim3(maxmoves, kMoveSlices), 256, 0, st>>>(eps, n, G, ptr, off, cnt, alpha, moves, stt, rq, lim, err,
                                                                 dirty);
  return cudaGetLastError();
}
cudaError_t launch_diff_positions(okmc_defect* d, const int* pos, int nd, Move* moves, DevState* stt, cudaStream_t st) {
  k_diff_positions<<<(nd + 127) / 128, 128, 0, st>>>(d, pos, nd, moves, stt);
  return cudaGetLastError();
}
cudaError_t launch_gather_positions(const okmc_defect* d, int* pos, int nd, cudaStream_t st) {
  k_gather_positions<<<(nd + 127) / 128, 128, 0, st>>>(d, pos, nd);
  return cudaGetLastError();
}
template <class Q, class T>
cudaError_t launch_fixed_to_real(const Q* eps, T* out, size_t total, double q, cudaStream_t st) {
  k_fixed_to_real<Q, T><<<1216, 256, 0, st>>>(eps, out, total, q);
  return cudaGetLastError();
}
template <class Q>
cudaError_t launch_wfields(Q* f, int3 n, const int* ptr, const int* off, const uint8_t* cnt, const WBatch& b, cudaStream_t st) {
  k_wfields<Q><<<2 * b.nb, 256, 0, st>>>(f, n, ptr, off, cnt, b);
  return cudaGetLastError();
}
template <class QT>
cudaError_t launch_qtable(QT* out, const PassCfg& c, const QTypes& qt, cudaStream_t st) {
  k_qtable<QT><<<1216, 256, 0, st>>>(out, c, qt);
  return cudaGetLastError();
}
template <class T>
cudaError_t launch_selfterm(const C2<T>* spec, const PassCfg& c, const WBatch& b, const T* qtab, const double2* phx,
                            const double2* phy, const double2* phz, double* partial, int nblocks, const double* alpha,
                            double pref, double* W, cudaStream_t st) {
  k_selfterm_partial<T, T><<<nblocks, 256, 0, st>>>(spec, c, b, qtab, phx, phy, phz, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_selfterm_final<<<1, 32, 0, st>>>(partial, nblocks, b, alpha, pref, W);
  return cudaGetLastError();
}
template <class T>
cudaError_t launch_energies(const T* sig, int3 n, const okmc_defect* d, const DefGeo* G, int nd, const int* ptr,
                            const int* off, const uint8_t* cnt, const double* alpha, const double* W, double pref,
                            int want_cand, const int* order, int nbig, double* E, double* Ec, RateArgs ra,
                            const DilatedLists& dl, cudaStream_t st) {
  if (nd == 0) return cudaSuccess;
  if (nbig < 0 || nbig > nd) return cudaErrorInvalidValue;
  constexpr int per = kEnergyThreads / 32;
  const int grid = nbig + (nd - nbig + per - 1) / per;
  k_energies<T><<<grid, kEnergyThreads, 0, st>>>(sig, n, d, G, ptr, off, cnt, alpha, W, pref, want_cand, order, E, Ec, ra,
                                                  dl, nd, nbig);
  return cudaGetLastError();
}
template <class T>
cudaError_t launch_energy_chunks(const T* sig, int3 n, const okmc_defect* d, const DefGeo* G, int nd,
                                 const DilatedLists& dl, const ChunkArgs& ca, cudaStream_t st) {
  if (nd == 0) return cudaSuccess;
  if (ca.nchunk <= 0) return cudaErrorInvalidValue;
  k_energy_chunks<T><<<(ca.nchunk + 7) / 8, 256, 0, st>>>(sig, n, d, G, dl, ca);
  return cudaGetLastError();
}
template cudaError_t launch_energy_chunks<float>(const float*, int3, const okmc_defect*, const DefGeo*, int,
                                                 const DilatedLists&, const ChunkArgs&, cudaStream_t);
template cudaError_t launch_energy_chunks<double>(const double*, int3, const okmc_defect*, const DefGeo*, int,
                                                  const DilatedLists&, const ChunkArgs&, cudaStream_t);
cudaError_t launch_energy_finish(const okmc_defect* d, const DefGeo* G, int nd, const DilatedLists& dl,
                                 const ChunkArgs& ca, const double* alpha, const double* W, double pref, double* E,
                                 double* Ec, RateArgs ra, cudaStream_t st) {
  if (nd == 0) return cudaSuccess;
  const int nq = (nd + 2) / 3;
  k_energy_finish<<<(nq + 1) / 2, 64, 0, st>>>(d, G, dl, ca, alpha, W, pref, nd, E, Ec, ra);
  return cudaGetLastError();
}
cudaError_t launch_residence(okmc_defect* d, int nd, const double* rates, const double* rsum, int3 n, uint64_t seed,
                             Move* moves, DevState* stt, cudaStream_t st) {
  k_residence<<<1, kEventThreads, 0, st>>>(d, nd, rates, rsum, n, (uint32_t)seed, (uint32_t)(seed >> 32), moves, stt);
  return cudaGetLastError();
}
cudaError_t launch_fixed_dt(okmc_defect* d, const DefGeo* G, int nd, const double* rates, double nu0, double kT, int3 n,
                            uint64_t seed, Move* moves, DevState* stt, cudaStream_t st) {
  k_fixed_dt<<<1, kEventThreads, 0, st>>>(d, G, nd, rates, nu0, kT, n, (uint32_t)seed, (uint32_t)(seed >> 32), moves, stt);
  return cudaGetLastError();
}

template cudaError_t launch_voxelise<int32_t>(int32_t*, int3, const okmc_defect*, const DefGeo*, int, const int*, const int*,
                                              const uint8_t*, const double*, double, double, int*, cudaStream_t);
template cudaError_t launch_voxelise<int64_t>(int64_t*, int3, const okmc_defect*, const DefGeo*, int, const int*, const int*,
                                              const uint8_t*, const double*, double, double, int*, cudaStream_t);
template cudaError_t launch_apply_moves<int32_t>(int32_t*, int3, const DefGeo*, int, const int*, const int*, const uint8_t*,
                                                 const double*, const Move*, const DevState*, double, double, int*, int*, cudaStream_t);
template cudaError_t launch_apply_moves<int64_t>(int64_t*, int3, const DefGeo*, int, const int*, const int*, const uint8_t*,
                                                 const double*, const Move*, const DevState*, double, double, int*, int*, cudaStream_t);
template cudaError_t launch_fixed_to_real<int32_t, float>(const int32_t*, float*, size_t, double, cudaStream_t);
template cudaError_t launch_fixed_to_real<int64_t, double>(const int64_t*, double*, size_t, double, cudaStream_t);
template cudaError_t launch_wfields<int32_t>(int32_t*, int3, const int*, const int*, const uint8_t*, const WBatch&, cudaStream_t);
template cudaError_t launch_wfields<int64_t>(int64_t*, int3, const int*, const int*, const uint8_t*, const WBatch&, cudaStream_t);
template cudaError_t launch_qtable<float>(float*, const PassCfg&, const QTypes&, cudaStream_t);
template cudaError_t launch_qtable<double>(double*, const PassCfg&, const QTypes&, cudaStream_t);
template cudaError_t launch_selfterm<float>(const C2<float>*, const PassCfg&, const WBatch&, const float*, const double2*,
                                           const double2*, const double2*, double*, int, const double*, double, double*,
                                           cudaStream_t);
template cudaError_t launch_selfterm<double>(const C2<double>*, const PassCfg&, const WBatch&, const double*, const double2*,
                                            const double2*, const double2*, double*, int, const double*, double, double*,
                                            cudaStream_t);
template cudaError_t launch_energies<float>(const float*, int3, const okmc_defect*, const DefGeo*, int, const int*, const int*,
                                           const uint8_t*, const double*, const double*, double, int, const int*, int,
                                           double*, double*, RateArgs, const DilatedLists&, cudaStream_t);
template cudaError_t launch_energies<double>(const double*, int3, const okmc_defect*, const DefGeo*, int, const int*,
                                            const int*, const uint8_t*, const double*, const double*, double, int, const int*,
                                            int, double*, double*, RateArgs, const DilatedLists&, cudaStream_t);

}  // namespace okmc
