// Fast FP32 solve passes for nx = ny and nz in {32, 48, 64, 96, 128, 160, 192, 256, 320}: the same three passes and data layout as solve.cu, with register
// line FFTs (fft_reg.cuh) instead of the generic shared-memory Stockham engine,
// loads issued a whole line (or a whole tile) ahead, and clusters sized so that
// two CTAs share each SM.
//
//   plane_fwd_fast : per (component, z) plane; rows of nx reals -> complex rows of
//                    nx/2 (8 or 4 threads per row, all loads of a row in flight),
//                    untangling, distributed-shared-memory scatter of the kx
//                    columns to their owner CTA, cluster barrier, column FFTs of
//                    length ny (in place, skewed exchange), contiguous stores.
//   pencil_fast    : per tile of 8 consecutive ky at one kx: the 6 x nz x 8 tile
//                    arrives by 16-byte cp.async that bypass L1 (all in flight at
//                    once) into a swizzled layout, forward z FFTs in place, Green
//                    operator, inverse z FFTs, stores.
//   plane_inv_fast : inverse of plane_fwd_fast.
#include <algorithm>
#include <cooperative_groups.h>
#include <type_traits>

#include "fft_reg.cuh"

namespace cg = cooperative_groups;

namespace okmc {

namespace {
constexpr int kT = 256;  // threads per CTA

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
// Split cluster barrier.  Every thread arrives once at its CTA's start and waits before
// its first store into another CTA's shared memory, which must be running by then (the
// CTAs of a cluster are launched together, so the wait ends at once); the closing
// cluster.sync() is the barrier's next phase.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory"); }
// hint: bring the 128-byte line holding p into L2 (no effect on results)
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p)); }
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
}  // namespace

template <int H, int NY>
__device__ __forceinline__ void load_tw(C2<float>* twH, C2<float>* twY, C2<float>* untw, const PassCfg& c) {
  fill_tw2<H>(twH, reinterpret_cast<const C2<float>*>(c.ftwH));
  fill_tw2<NY>(twY, reinterpret_cast<const C2<float>*>(c.ftwY));
  const C2<float>* gU = reinterpret_cast<const C2<float>*>(c.ftwU);
  for (int i = threadIdx.x; i <= H; i += blockDim.x) untw[i] = gU[i];
}

// Twiddle tables of a plane pass at the start of its shared memory, padded to a whole
// number of 16-byte units so that every buffer after them stays 16-byte aligned
template <int H, int NY>
__host__ __device__ constexpr size_t plane_tw_bytes() {
  return (sizeof(C2<float>) * ((size_t)tw2_size<H>() + tw2_size<NY>() + H + 1) + 15) / 16 * 16;
}

// The twiddle tables of a plane pass staged through registers (at most a few values per
// thread): load() first, so that these L2 hits are not queued behind the pass's first
// DRAM loads, store() once those are in flight.
template <int H, int NY, int NTHR>
struct TwStage {
  static constexpr int NH = (tw2_size<H>() + NTHR - 1) / NTHR, NYs = (tw2_size<NY>() + NTHR - 1) / NTHR;
  static constexpr int NU = (H + 1 + NTHR - 1) / NTHR;
  C2<float> h[NH], y[NYs], u[NU];
  __device__ __forceinline__ void load(const PassCfg& c, int tid) {
    const C2<float>* gH = reinterpret_cast<const C2<float>*>(c.ftwH);
    const C2<float>* gY = reinterpret_cast<const C2<float>*>(c.ftwY);
    const C2<float>* gU = reinterpret_cast<const C2<float>*>(c.ftwU);
#pragma unroll
    for (int j = 0; j < NH; ++j)
      if (tid + NTHR * j < tw2_size<H>()) h[j] = tw2_entry<H>(gH, tid + NTHR * j);
#pragma unroll
    for (int j = 0; j < NYs; ++j)
      if (tid + NTHR * j < tw2_size<NY>()) y[j] = tw2_entry<NY>(gY, tid + NTHR * j);
#pragma unroll
    for (int j = 0; j < NU; ++j)
      if (tid + NTHR * j <= H) u[j] = gU[tid + NTHR * j];
  }
  __device__ __forceinline__ void store(C2<float>* twH, C2<float>* twY, C2<float>* untw, int tid) const {
#pragma unroll
    for (int j = 0; j < NH; ++j)
      if (tid + NTHR * j < tw2_size<H>()) twH[tid + NTHR * j] = h[j];
#pragma unroll
    for (int j = 0; j < NYs; ++j)
      if (tid + NTHR * j < tw2_size<NY>()) twY[tid + NTHR * j] = y[j];
#pragma unroll
    for (int j = 0; j < NU; ++j)
      if (tid + NTHR * j <= H) untw[tid + NTHR * j] = u[j];
  }
};

// Row of a plane handled by row group g in the row phases of the inverse pass.  A row
// buffer stride of H + 1 complex puts adjacent rows 2 banks apart, so two groups of
// one half-warp on adjacent rows collide; groups of one half-warp take rows NTH apart
// instead (their 64-bit accesses then cover the 32 banks once).  A bijection on each
// block of 16 rows.
template <int NTH>
__device__ __forceinline__ int row_of_group(int g) {
  constexpr int q = 16 / NTH;  // groups per half-warp
  const int hw = g / q, i = g % q;
  return (hw / NTH) * 16 + (hw % NTH) + i * NTH;
}

// ---------------------------------------------------------------- plane passes
// One cluster of CS CTAs (256 threads, two CTAs per SM) per (component, z) plane.
// Rows: a group of reg_nt<H> threads per row, all of a row's loads in flight,
// untangling, distributed-shared-memory scatter of every kx value to its column
// owner; column 0 carries (X[0], X[nx/2]) packed so that every CTA owns exactly
// H/CS columns.  Columns: in place in shared memory, contiguous stores.
constexpr int kNT = 256;

template <int H, int NY>
struct NShape {
  static constexpr int NTH = reg_nt<H>(), GR = kNT / NTH;
  static constexpr int NTY = reg_nt<NY>(), GC = kNT / NTY;
  static constexpr int R2H = RegPlan<H>::R2, R2Y = RegPlan<NY>::R2;
  static constexpr int XS = RegPlan<H>::R1 * (R2H + 1);       // row exchange slots
  static constexpr int XSY = RegPlan<NY>::R1 * (R2Y + 1);     // column exchange slots
  static constexpr int XB = GR * XS > GC * XSY ? GR * XS : GC * XSY;
  // inverse pass: column groups XSY + 1 apart (odd, so that a row of the staged column
  // outputs, one element per group, is read without bank conflicts)
  static constexpr int XSYP = XSY + 1;
  static constexpr int XBI = GR * XS > GC * XSYP ? GR * XS : GC * XSYP;
  static constexpr int LDC = NY + 1, LDR = H + 1;
};
template <int H, int NY>
__host__ __device__ constexpr size_t nfwd_smem(int cs) {
  using S = NShape<H, NY>;
  return plane_tw_bytes<H, NY>() + sizeof(C2<float>) * ((size_t)(H / cs) * S::LDC + (size_t)S::GR * S::XS);
}
template <int H, int NY>
__host__ __device__ constexpr size_t ninv_smem(int cs, int wide = 0) {
  using S = NShape<H, NY>;
  return plane_tw_bytes<H, NY>() + sizeof(C2<float>) * ((size_t)(NY / cs) * (wide == 2 ? H + 2 : S::LDR) + (size_t)S::XBI);
}

// store v at column k, row y of the column buffer of the CTA that owns column k
template <int CS, int CPER, int LDC>
__device__ __forceinline__ void put_col(cg::cluster_group& cluster, C2<float>* col, int h, int k, int y, C2<float> v) {
  const int owner = k / CPER;
  C2<float>* base = (CS > 1 && owner != h) ? cluster.map_shared_rank(col, owner) : col;
  base[(k % CPER) * LDC + y] = v;
}

// One (component, z) plane of the forward pass, by the CS CTAs of a cluster (cluster
// rank h); smem_raw: nfwd_smem<H, NY>(CS) bytes of dynamic shared memory.  A clean plane
// (dirty flag 0) returns at once in every CTA of the cluster alike.
// pf > 0: first bring into L2 this CTA's rows of plane + pf (when that plane is dirty),
// the plane whose cluster will most likely take this one's place a wave later.
template <int H, int NY, int CS>
__device__ __forceinline__ void plane_fwd_item(const int32_t* __restrict__ eps, C2<float>* __restrict__ spec,
                                               const PassCfg& c, int plane, unsigned char* smem_raw, int pf = 0,
                                               int nplanes = 0) {
  using S = NShape<H, NY>;
  constexpr int CPER = H / CS, ROWS = NY / CS;
  C2<float>* twH = reinterpret_cast<C2<float>*>(smem_raw);
  C2<float>* twY = twH + tw2_size<H>();
  C2<float>* untw = twY + tw2_size<NY>();
  unsigned char* after_tw = smem_raw + plane_tw_bytes<H, NY>();
  C2<float>* col = reinterpret_cast<C2<float>*>(after_tw);  // [CPER][LDC]
  C2<float>* xb = col + CPER * S::LDC;                            // [GR][XS]
  cg::cluster_group cluster = cg::this_cluster();
  const int h = CS > 1 ? (int)cluster.block_rank() % CS : 0;
  // a plane whose eigenstrain has not changed keeps its transform from the last pass
  // (every CTA of the cluster reads the same flag, so the whole cluster leaves)
  if (c.dirty && c.dirty[plane] == 0) return;
  if (CS > 1) cluster_arrive();
  const int tid = threadIdx.x;
  if (pf > 0 && plane + pf < nplanes && (!c.dirty || c.dirty[plane + pf] != 0)) {
    const char* nx_rows = reinterpret_cast<const char*>(eps + ((size_t)(plane + pf) * NY + (size_t)h * ROWS) * (2 * H));
    for (int i = tid; i < ROWS * 2 * H * 4 / 128; i += kNT) prefetch_l2(nx_rows + (size_t)i * 128);
  }
  const size_t P = (size_t)(H + 1) * NY;
  const float q = (float)c.q;
  const int g = tid / S::NTH, t = tid % S::NTH;
  // loads of row group r0 (the first group's loads fly while the twiddles are filled)
  RegLine<H> line;
  auto load_rows = [&](int r0) {
    const bool act = r0 + g < ROWS;
    const int y = h * ROWS + (act ? r0 + g : 0);
    const int2* row = reinterpret_cast<const int2*>(eps + ((size_t)plane * NY + y) * (2 * H));
    reg_load<H>(line, [&](int i) {
      const int2 v = __ldg(row + i);
      return C2<float>{__int2float_rn(v.x) * q, __int2float_rn(v.y) * q};
    }, t, act);
  };
  TwStage<H, NY, kNT> tws;
  tws.load(c, tid);
  load_rows(0);
  tws.store(twH, twY, untw, tid);
  __syncthreads();
  {  // rows along x
    C2<float>* xg = xb + g * S::XS;
    for (int r0 = 0; r0 < ROWS; r0 += S::GR) {
      const bool act = r0 + g < ROWS;
      const int y = h * ROWS + (act ? r0 + g : 0);
      if (r0 > 0) load_rows(r0);
      auto st = [&](int k, C2<float> v) { xg[k] = v; };
      reg_fft_loaded<false, H>(line, XPad<S::R2H>{xg}, st, twH, t, act);
      if (CS > 1 && r0 == 0) cluster_wait();
      if (act) {
        // X[k] = (A + B)/2 - (i/2) w^k (A - B) and X[H-k] = conj((A + B)/2) - (i/2) w^(H-k) conj(B - A)
        // from the same A = Z[k], B = conj Z[H-k]; k = 0 packs (X[0], X[nx/2])
#pragma unroll
        for (int j = 0; j <= H / 2 / S::NTH; ++j) {
          const int k = t + S::NTH * j;
          if (k > H / 2) break;
          const C2<float> A = xg[k];
          if (k == 0) {
            put_col<CS, CPER, S::LDC>(cluster, col, h, 0, y, C2<float>{A.x + A.y, A.x - A.y});
            continue;
          }
          const C2<float> B = conjg(xg[H - k]);
          const C2<float> sum = A + B, d1 = cmul_rn(untw[k], A - B);
          put_col<CS, CPER, S::LDC>(cluster, col, h, k, y, C2<float>{0.5f * (sum.x + d1.y), 0.5f * (sum.y - d1.x)});
          if (2 * k != H) {
            // w^(H-k) = -conj(w^k), so w^(H-k) conj(B - A) = conj(w^k (A - B)) = conj(d1)
            const C2<float> d2 = conjg(d1);
            put_col<CS, CPER, S::LDC>(cluster, col, h, H - k, y,
                                      C2<float>{0.5f * (sum.x + d2.y), 0.5f * (-sum.y - d2.x)});
          }
        }
      }
      __syncwarp();
    }
  }
  if (CS > 1) cluster.sync();
  else __syncthreads();
  // every CTA of the cluster has read the flag before the barrier above
  if (c.dirty && h == 0 && tid == 0) c.dirty[plane] = 0;
  {  // columns along y
    const int g = tid / S::NTY, t = tid % S::NTY;
    for (int c0 = 0; c0 < CPER; c0 += S::GC) {
      const bool act = c0 + g < CPER;
      const int cc = act ? c0 + g : 0;
      const int kx = h * CPER + cc;
      C2<float>* cp = col + cc * S::LDC;
      C2<float>* out = spec + (size_t)plane * P + (size_t)kx * NY;
      const bool packed = (kx == 0);
      auto ld = [&](int i) { return cp[i]; };
      auto st = [&](int k, C2<float> v) {
        if (packed) cp[k] = v;
        else out[k] = v;
      };
      reg_fft<false, NY>(ld, XSkew<S::R2Y>{cp, 1}, st, twY, t, act);
      if (act && packed) {
        // P = A + i B, A and B the spectra of the real columns X[0] and X[nx/2]
        for (int k = t; k < NY; k += S::NTY) {
          const C2<float> Pk = cp[k], Pm = conjg(cp[k == 0 ? 0 : NY - k]);
          const C2<float> s = Pk + Pm, d = Pk - Pm;
          out[k] = C2<float>{0.5f * s.x, 0.5f * s.y};
          out[(size_t)H * NY + k] = C2<float>{0.5f * d.y, -0.5f * d.x};
        }
      }
    }
  }
}

template <int H, int NY, int CS>
__global__ void __launch_bounds__(kNT, 2) k_plane_fwd_n(const int32_t* __restrict__ eps, C2<float>* __restrict__ spec,
                                                        PassCfg c, int pf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  plane_fwd_item<H, NY, CS>(eps, spec, c, blockIdx.y, smem_raw, pf, gridDim.y);
}

// pf > 0: first bring into L2 this CTA's columns of plane + pf, the plane whose
// cluster will most likely take this one's place one wave later (pf = clusters
// resident at once), so that the next wave's loads hit L2 while this wave transforms.
// WIDE: each column group's transform output is staged in the group's own exchange
// slots, and after a barrier the CTA copies it out by rows: a warp then writes 16 or
// more consecutive kx of one row of the owner's buffer (128 contiguous bytes or more)
// instead of two kx of 16 rows.  Remote stores into another CTA's shared memory cost
// by the write pattern: the wide copy-out makes the scatter far cheaper.
// WIDE 2: as 1, with rows H + 2 apart (16-byte aligned), so that a lane of the copy-out
// carries two adjacent kx in one 16-byte store; the row phase then pairs the line
// groups of a half-warp on rows 4 apart (with lines of 8 threads; rows 8 apart would
// fall on the same banks at this pitch).
// One plane of the inverse pass by the CS CTAs of a cluster; nplanes bounds the L2
// prefetch of plane + pf (pf = 0: none).
template <int H, int NY, int CS, int WIDE>
__device__ __forceinline__ void plane_inv_item(const C2<float>* __restrict__ spec, float* __restrict__ sig,
                                               const PassCfg& c, int plane, int pf, int nplanes,
                                               unsigned char* smem_raw) {
  using S = NShape<H, NY>;
  constexpr int CPER = H / CS, ROWS = NY / CS;
  constexpr int LDR = WIDE == 2 ? H + 2 : S::LDR;
  static_assert(WIDE != 2 || S::NTH == 8, "the 16-byte copy-out pairs rows for lines of 8 threads");
  C2<float>* twH = reinterpret_cast<C2<float>*>(smem_raw);
  C2<float>* twY = twH + tw2_size<H>();
  C2<float>* untw = twY + tw2_size<NY>();
  unsigned char* after_tw = smem_raw + plane_tw_bytes<H, NY>();
  C2<float>* rowb = reinterpret_cast<C2<float>*>(after_tw);  // [ROWS][LDR]
  C2<float>* xb = rowb + ROWS * LDR;
  cg::cluster_group cluster = cg::this_cluster();
  const int h = CS > 1 ? (int)cluster.block_rank() % CS : 0;
  const int tid = threadIdx.x;
  const size_t P = (size_t)(H + 1) * NY;
  if (CS > 1) cluster_arrive();
  if (pf > 0 && plane + pf < nplanes) {
    const char* nx = reinterpret_cast<const char*>(spec + (size_t)(plane + pf) * P + (size_t)h * CPER * NY);
    for (int i = tid; i < CPER * NY * 8 / 128; i += kNT) prefetch_l2(nx + (size_t)i * 128);
    if (h == 0) {
      const char* nq = reinterpret_cast<const char*>(spec + (size_t)(plane + pf) * P + (size_t)H * NY);
      for (int i = tid; i < NY * 8 / 128; i += kNT) prefetch_l2(nq + (size_t)i * 128);
    }
  }
  {  // inverse columns along y, scattered to the row owners
    const int g = tid / S::NTY, t = tid % S::NTY;
    // loads of column group c0 (the first group's loads fly while the twiddles are filled)
    RegLine<NY> line;
    auto load_cols = [&](int c0) {
      const bool act = c0 + g < CPER;
      const int kx = h * CPER + (act ? c0 + g : 0);
      const C2<float>* in = spec + (size_t)plane * P + (size_t)kx * NY;
      const C2<float>* nyq = spec + (size_t)plane * P + (size_t)H * NY;
      const bool packed = (kx == 0);
      reg_load<NY>(line, [&](int i) {
        const C2<float> A = in[i];
        if (!packed) return A;
        const C2<float> B = nyq[i];
        return C2<float>{A.x - B.y, A.y + B.x};  // A + i B
      }, t, act);
    };
    TwStage<H, NY, kNT> tws;
    tws.load(c, tid);
    load_cols(0);
    tws.store(twH, twY, untw, tid);
    __syncthreads();
    C2<float>* xg = xb + g * (WIDE ? S::XSYP : S::XSY);
    for (int c0 = 0; c0 < CPER; c0 += S::GC) {
      const bool act = c0 + g < CPER;
      const int kx = h * CPER + (act ? c0 + g : 0);
      if (WIDE == 0 && c0 > 0) load_cols(c0);
      if constexpr (WIDE != 0) {
        auto st = [&](int k, C2<float> v) { xg[k] = v; };
        reg_fft_loaded<true, NY>(line, XPad<S::R2Y>{xg}, st, twY, t, act);
        // the next group's loads fly during the copy-out and its barriers
        if (c0 + S::GC < CPER) load_cols(c0 + S::GC);
        __syncthreads();
        if (CS > 1 && c0 == 0) cluster_wait();
        constexpr int GC = S::GC;
        const int ncol = CPER - c0 < GC ? CPER - c0 : GC;
        if constexpr (WIDE == 1) {
          for (int e = tid; e < NY * GC; e += kNT) {  // element (row k, column j)
            const int j = e % GC, k = e / GC;
            if (j < ncol) {
              const int owner = k / ROWS;
              C2<float>* base = (CS > 1 && owner != h) ? cluster.map_shared_rank(rowb, owner) : rowb;
              base[(k % ROWS) * LDR + h * CPER + c0 + j] = xb[j * S::XSYP + k];
            }
          }
        } else {
          // columns j, j + 1 of row k in one 16-byte store (h * CPER + c0, ncol and GC are
          // even, and rows start on 16-byte boundaries)
          for (int e = tid; e < NY * (GC / 2); e += kNT) {
            const int j = 2 * (e % (GC / 2)), k = e / (GC / 2);
            if (j < ncol) {
              const int owner = k / ROWS;
              C2<float>* base = (CS > 1 && owner != h) ? cluster.map_shared_rank(rowb, owner) : rowb;
              const C2<float> v0 = xb[j * S::XSYP + k], v1 = xb[(j + 1) * S::XSYP + k];
              *reinterpret_cast<float4*>(base + (k % ROWS) * LDR + h * CPER + c0 + j) = make_float4(v0.x, v0.y, v1.x, v1.y);
            }
          }
        }
        __syncthreads();
      } else {
        auto st = [&](int k, C2<float> v) {
          const int owner = k / ROWS;
          C2<float>* base = (CS > 1 && owner != h) ? cluster.map_shared_rank(rowb, owner) : rowb;
          base[(k % ROWS) * LDR + kx] = v;
        };
        if (CS > 1 && c0 == 0) cluster_wait();
        reg_fft_loaded<true, NY>(line, XPad<S::R2Y>{xg}, st, twY, t, act);
      }
    }
  }
  if (CS > 1) cluster.sync();
  else __syncthreads();
  {  // rows along x
    const int g = tid / S::NTH, t = tid % S::NTH;
    for (int r0 = 0; r0 < ROWS; r0 += S::GR) {
      // WIDE 2: the two groups of a half-warp on rows 4 apart (a bijection on each block of 8)
      const int yr = r0 + (WIDE == 2 ? (g >> 3) * 8 + ((g >> 1) & 3) + (g & 1) * 4 : row_of_group<S::NTH>(g));
      const bool act = yr < ROWS;
      const int yl = act ? yr : 0;
      C2<float>* R = rowb + yl * LDR;
      auto ld = [&](int k) {
        if (k == 0) {
          const C2<float> p = R[0];
          return C2<float>{p.x + p.y, p.x - p.y};
        }
        const C2<float> Xk = R[k], Xc = conjg(R[H - k]);
        const C2<float> E = Xk + Xc;
        const C2<float> O = cmul_rn(conjg(untw[k]), Xk - Xc);
        return C2<float>{E.x - O.y, E.y + O.x};
      };
      C2<float>* orow = reinterpret_cast<C2<float>*>(sig + ((size_t)plane * NY + h * ROWS + yl) * (2 * H));
      auto st = [&](int k, C2<float> v) { orow[k] = v; };
      reg_fft<true, H>(ld, XSkew<S::R2H>{R, 1}, st, twH, t, act);
    }
  }
}

template <int H, int NY, int CS, int WIDE>
__global__ void __launch_bounds__(kNT, 2) k_plane_inv_n(const C2<float>* __restrict__ spec, float* __restrict__ sig,
                                                        PassCfg c, int pf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  plane_inv_item<H, NY, CS, WIDE>(spec, sig, c, blockIdx.y, pf, gridDim.y, smem_raw);
}

// Staged variant of the inverse plane pass: the CTA's CPER columns are one contiguous
// block of the kx-major spectrum plane, so they arrive by 16-byte cp.async at the
// start (no registers held while the copies fly; the owner of column 0 also fetches
// the Nyquist column), and each column is transformed in place in the staging
// buffer, with no separate exchange buffer.  The row phase is the same as above.
template <int H, int NY>
__host__ __device__ constexpr size_t sinv_smem(int cs) {
  return plane_tw_bytes<H, NY>() + sizeof(C2<float>) * ((size_t)(H / cs + 1) * NY + (size_t)(NY / cs) * (H + 1));
}

template <int H, int NY, int CS, int NTHR, int MINB>
__global__ void __launch_bounds__(NTHR, MINB) k_plane_inv_s(const C2<float>* __restrict__ spec, float* __restrict__ sig,
                                                         PassCfg c) {
  constexpr int CPER = H / CS, ROWS = NY / CS, LDR = H + 1;
  constexpr int NTY = reg_nt<NY>(), GC = NTHR / NTY, NTH = reg_nt<H>(), GR = NTHR / NTH;
  constexpr int R2Y = RegPlan<NY>::R2, R2H = RegPlan<H>::R2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<float>* twH = reinterpret_cast<C2<float>*>(smem_raw);
  C2<float>* twY = twH + tw2_size<H>();
  C2<float>* untw = twY + tw2_size<NY>();
  unsigned char* after_tw = smem_raw + plane_tw_bytes<H, NY>();
  C2<float>* stg = reinterpret_cast<C2<float>*>(after_tw);  // [CPER][NY] own columns, then [NY] Nyquist
  C2<float>* nyq = stg + CPER * NY;
  C2<float>* rowb = nyq + NY;                                     // [ROWS][LDR]
  cg::cluster_group cluster = cg::this_cluster();
  const int h = CS > 1 ? (int)cluster.block_rank() : 0;
  const int plane = blockIdx.y;
  const int tid = threadIdx.x;
  if (CS > 1) cluster_arrive();
  const size_t P = (size_t)(H + 1) * NY;
  {
    const C2<float>* src = spec + (size_t)plane * P + (size_t)h * CPER * NY;
    for (int i = tid; i < CPER * NY / 2; i += NTHR) cp_async16(stg + 2 * i, src + 2 * i);
    if (h == 0) {
      const C2<float>* sn = spec + (size_t)plane * P + (size_t)H * NY;
      for (int i = tid; i < NY / 2; i += NTHR) cp_async16(nyq + 2 * i, sn + 2 * i);
    }
  }
  load_tw<H, NY>(twH, twY, untw, c);
  cp_async_wait_all();
  __syncthreads();
  if (CS > 1) cluster_wait();
  {  // inverse columns along y, in place, scattered to the row owners
    const int g = tid / NTY, t = tid % NTY;
    for (int c0 = 0; c0 < CPER; c0 += GC) {
      const bool act = c0 + g < CPER;
      const int cc = act ? c0 + g : 0;
      const int kx = h * CPER + cc;
      C2<float>* col = stg + cc * NY;
      const bool packed = (kx == 0);
      auto ld = [&](int i) {
        const C2<float> A = col[i];
        if (!packed) return A;
        const C2<float> B = nyq[i];
        return C2<float>{A.x - B.y, A.y + B.x};  // A + i B
      };
      auto st = [&](int k, C2<float> v) {
        const int owner = k / ROWS;
        C2<float>* base = (CS > 1 && owner != h) ? cluster.map_shared_rank(rowb, owner) : rowb;
        base[(k % ROWS) * LDR + kx] = v;
      };
      reg_fft<true, NY>(ld, XSkew<R2Y>{col, 1}, st, twY, t, act);
    }
  }
  if (CS > 1) cluster.sync();
  else __syncthreads();
  {  // rows along x
    const int g = tid / NTH, t = tid % NTH;
    for (int r0 = 0; r0 < ROWS; r0 += GR) {
      const int yr = r0 + row_of_group<NTH>(g);
      const bool act = yr < ROWS;
      const int yl = act ? yr : 0;
      C2<float>* R = rowb + yl * LDR;
      auto ld = [&](int k) {
        if (k == 0) {
          const C2<float> p = R[0];
          return C2<float>{p.x + p.y, p.x - p.y};
        }
        const C2<float> Xk = R[k], Xc = conjg(R[H - k]);
        const C2<float> E = Xk + Xc;
        const C2<float> O = cmul_rn(conjg(untw[k]), Xk - Xc);
        return C2<float>{E.x - O.y, E.y + O.x};
      };
      C2<float>* orow = reinterpret_cast<C2<float>*>(sig + ((size_t)plane * NY + h * ROWS + yl) * (2 * H));
      auto st = [&](int k, C2<float> v) { orow[k] = v; };
      reg_fft<true, H>(ld, XSkew<R2H>{R, 1}, st, twH, t, act);
    }
  }
}

constexpr int kTW = 8;
constexpr int kLDT = kTW + 1;  // padded row of a tile: conflict-free strided line access

// Tile layouts.  Padded: rows of kLDT complex, element (row, col) at row * kLDT + col.
// Swizzled: dense rows of kTW = 8 complex (64 bytes, so every row starts on a 16-byte
// boundary and arrives by 16-byte copies that bypass L1), with the 16-byte pieces of a
// row permuted by bits 1-2 of the row: element (row, col) at row * 8 + (col ^ (row & 6)).
// A half-warp then reads 8 consecutive rows of each of two lines of opposite column
// parity without bank conflicts.
template <int NZ, bool SWZ>
__host__ __device__ constexpr size_t pencil_fast_smem() {
  return (sizeof(C2<float>) * (size_t)tw2_size<NZ>() + 15) / 16 * 16 + sizeof(C2<float>) * ((size_t)6 * NZ * (SWZ ? kTW : kLDT));
}
template <bool SWZ>
__device__ __forceinline__ int tile_at(int row, int col) {
  return SWZ ? row * kTW + (col ^ (row & 6)) : row * kLDT + col;
}

// Exchange slots of a line of the swizzled tile (the skew of XSkew, rows r0 + n1 * R2 + m).
// With m = k2 XOR n1 (R2 = 16), the eight lanes of a line in a half-warp still meet all
// eight values of m mod 8, as with the additive skew, so the two lines of opposite
// column parity that share the half-warp stay on disjoint banks.
template <int R2>
struct XSwz {
  C2<float>* tile;
  int r0, col;
  __device__ __forceinline__ C2<float>& operator()(int n1, int k2) const {  // n1 < R2
    return tile[tile_at<true>(r0 + n1 * R2 + xskew<R2>(n1, k2), col)];
  }
};

// Tile row handled by row counter r in the load, Green and store loops of the padded
// tile: lanes 0-7 and 8-15 of a half-warp take rows 8 apart, whose 18-word stride puts
// them 16 banks apart (adjacent rows would wrap onto the same banks).  A bijection on
// each block of 16 rows; NZ is a multiple of 16, so a block never straddles two
// components.  The swizzled tile takes adjacent rows (row & 1 selects the bank half).
__device__ __forceinline__ int tile_row(int r) { return (r & ~15) + ((r & 1) << 3) + ((r >> 1) & 7); }

// in and out may be the same buffer: every CTA reads its whole tile before it writes.
// SWZ false: padded tile, 8-byte copies (through L1).  SWZ true: swizzled tile, every
// row by 16-byte copies that bypass L1; with lines of 16 threads the groups of a warp
// are paired so that each half-warp holds 8 threads of each of two adjacent lines.  The
// two layouts give the same arithmetic.  (8-byte copies allocate in L1, which two CTAs'
// shared memory leave small, and so limit the loads in flight on the SM.)
// Forward z FFTs, Green operator and inverse z FFTs of one tile (8 consecutive ky at one
// kx, every kz, six components) held in shared memory in layout SWZ; ends on a barrier.
template <int NZ, bool SWZ>
__device__ __forceinline__ void pencil_tile(C2<float>* tile, const C2<float>* twZ, const PassCfg& c, int kx, int ky0) {
  const int tid = threadIdx.x;
  constexpr int NTZ = reg_nt<NZ>(), GL = kT / NTZ, R2Z = RegPlan<NZ>::R2;
  int g = tid / NTZ, t = tid % NTZ;
  if (SWZ && NTZ == 16) {  // group 2w + b of warp w: lanes 8b + {0-7, 16-23}
    g = 2 * (tid >> 5) + ((tid >> 3) & 1);
    t = (tid & 7) | (((tid >> 4) & 1) << 3);
  }
  auto lines = [&](auto inv) {
    constexpr bool INV = decltype(inv)::value;
    for (int l0 = 0; l0 < 6 * kTW; l0 += GL) {
      const bool act = l0 + g < 6 * kTW;
      const int l = act ? l0 + g : 0;
      const int r0 = (l / kTW) * NZ, col = l % kTW;
      if constexpr (SWZ) {
        auto ld = [&](int i) { return tile[tile_at<true>(r0 + i, col)]; };
        auto st = [&](int k, C2<float> v) { tile[tile_at<true>(r0 + k, col)] = v; };
        reg_fft<INV, NZ>(ld, XSwz<R2Z>{tile, r0, col}, st, twZ, t, act);
      } else {
        C2<float>* base = tile + r0 * kLDT + col;
        auto ld = [&](int i) { return base[i * kLDT]; };
        auto st = [&](int k, C2<float> v) { base[k * kLDT] = v; };
        reg_fft<INV, NZ>(ld, XSkew<R2Z>{base, kLDT}, st, twZ, t, act);
      }
    }
  };
  auto row_of = [](int r) { return SWZ ? r : tile_row(r); };
  lines(std::false_type{});
  __syncthreads();
  if (!c.forward_only) {
    const float scale = 1.0f / ((float)c.nx * (float)c.ny * (float)c.nz);
    for (int idx = tid; idx < kTW * NZ; idx += kT) {
      const int t8 = idx & (kTW - 1), kz = row_of(idx >> 3);
      C2<float> e[6];
#pragma unroll
      for (int a = 0; a < 6; ++a) e[a] = tile[tile_at<SWZ>(a * NZ + kz, t8)];
      green_point<float>(e, kx, ky0 + t8, kz, c, scale);
#pragma unroll
      for (int a = 0; a < 6; ++a) tile[tile_at<SWZ>(a * NZ + kz, t8)] = e[a];
    }
    __syncthreads();
    lines(std::true_type{});
    __syncthreads();
  }
}

// One tile of the pencil pass, staged by per-thread asynchronous copies.
template <int NZ, bool SWZ>
__device__ __forceinline__ void pencil_item(const C2<float>* in, C2<float>* out, const PassCfg& c, int tile_index,
                                            unsigned char* smem_raw) {
  C2<float>* twZ = reinterpret_cast<C2<float>*>(smem_raw);
  C2<float>* tile = reinterpret_cast<C2<float>*>(smem_raw + (sizeof(C2<float>) * tw2_size<NZ>() + 15) / 16 * 16);  // [comp * NZ + kz][8 or 9]
  const int tid = threadIdx.x;
  const size_t P = (size_t)(c.H + 1) * c.ny;
  const size_t p0 = (size_t)tile_index * kTW;
  const int kx = (int)(p0 / c.ny), ky0 = (int)(p0 % c.ny);
  if constexpr (SWZ) {
    for (int idx = tid; idx < 6 * NZ * 4; idx += kT) {  // four 16-byte pieces per row
      const int row = idx >> 2, t = 2 * (idx & 3);
      cp_async16(tile + tile_at<true>(row, t), in + (size_t)row * P + p0 + t);
    }
  } else {
    for (int idx = tid; idx < 6 * NZ * kTW; idx += kT) {
      const int t = idx & (kTW - 1), row = tile_row(idx >> 3);  // row = comp * NZ + kz
      cp_async8(tile + row * kLDT + t, in + (size_t)row * P + p0 + t);
    }
  }
  fill_tw2<NZ>(twZ, reinterpret_cast<const C2<float>*>(c.ftwZ));
  cp_async_wait_all();
  __syncthreads();
  pencil_tile<NZ, SWZ>(tile, twZ, c, kx, ky0);
  for (int idx = tid; idx < 6 * NZ * kTW; idx += kT) {
    const int t8 = idx & (kTW - 1), row = SWZ ? idx >> 3 : tile_row(idx >> 3);
    out[(size_t)row * P + p0 + t8] = tile[tile_at<SWZ>(row, t8)];
  }
}

// ---- tensor-memory-access (TMA) staging of the pencil tile
// The spectra seen as a 2-D float tensor of 6 * nz rows (row comp * nz + kz) of 2 * P
// floats; a box is 16 floats (one tile row of 8 complex, 64 bytes) wide and TmaBox<NZ>
// rows high, and the 64-byte swizzle of the tensor map lays it out exactly as
// tile_at<true> (16-byte piece j of row r at piece j ^ ((r >> 1) & 3)) when the tile
// starts on a 1024-byte boundary.
template <int NZ>
struct TmaBox {
  static constexpr int BH = NZ <= 256 ? NZ : NZ / 2;  // a box spans at most 256 rows
  static constexpr int NB = 6 * NZ / BH;
  static constexpr unsigned kBytes = 6u * NZ * kTW * sizeof(C2<float>);
};
static_assert(TmaBox<320>::BH * 2 == 320 && TmaBox<320>::kBytes < (1u << 20), "box split / tx-count range");

template <int NZ>
__host__ __device__ constexpr size_t pencil_tma_smem() {
  // twiddles, mbarrier (16 bytes), up to 1023 bytes to reach a 1024-byte boundary, tile
  return (sizeof(C2<float>) * (size_t)tw2_size<NZ>() + 15) / 16 * 16 + 16 + 1023 + TmaBox<NZ>::kBytes;
}

namespace {
constexpr unsigned long long kBulkWaitNs = 500000000ull;  // 0.5 s: a copy that slow has failed

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// Wait for phase `parity` of the mbarrier to complete, giving up after kBulkWaitNs.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0; it < (1u << 28); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 31) == 31 && global_ns() - t0 > kBulkWaitNs) return false;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int x, int y, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, unsigned src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(map), "r"(x), "r"(y),
               "r"(src)
               : "memory");
}
}  // namespace

// One tile of the pencil pass, staged by TMA: one thread issues the tile's box loads onto
// an mbarrier that every thread then waits on (bounded: on timeout the CTA records error
// 6, waits once more, bounded, for the copies in flight, and returns without output);
// after the transforms one thread stores the boxes back and waits until they have been
// read out of shared memory.
template <int NZ>
__device__ __forceinline__ void pencil_item_tma(const CUtensorMap* tin, const CUtensorMap* tout, const PassCfg& c,
                                                int tile_index, unsigned char* smem_raw) {
  using B = TmaBox<NZ>;
  constexpr unsigned TWB = (sizeof(C2<float>) * tw2_size<NZ>() + 15) / 16 * 16;
  C2<float>* twZ = reinterpret_cast<C2<float>*>(smem_raw);
  const unsigned s0 = (unsigned)__cvta_generic_to_shared(smem_raw);
  const unsigned bar = s0 + TWB;
  const unsigned ts = (s0 + TWB + 16 + 1023) & ~1023u;
  C2<float>* tile = reinterpret_cast<C2<float>*>(smem_raw + (ts - s0));
  const int tid = threadIdx.x;
  const int p0 = tile_index * kTW;
  const int kx = p0 / c.ny, ky0 = p0 % c.ny;
  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(bar, B::kBytes + (unsigned)c.tx_extra);
#pragma unroll 1
    for (int b = 0; b < B::NB; ++b) tma_load_2d(ts + (unsigned)b * B::BH * 64u, tin, 2 * p0, b * B::BH, bar);
  }
  fill_tw2<NZ>(twZ, reinterpret_cast<const C2<float>*>(c.ftwZ));
  const bool ok = mbar_wait_bounded(bar, 0);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      atomicExch(c.err, 6);
      mbar_wait_bounded(bar, 0);
    }
    return;
  }
  pencil_tile<NZ, true>(tile, twZ, c, kx, ky0);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // the tile's writes, visible to the bulk copies
  __syncthreads();
  if (tid == 0) {
#pragma unroll 1
    for (int b = 0; b < B::NB; ++b) tma_store_2d(tout, 2 * p0, b * B::BH, ts + (unsigned)b * B::BH * 64u);
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
  }
}

template <int NZ>
__global__ void __launch_bounds__(kT, 2)
    k_pencil_tma(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout, PassCfg c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pencil_item_tma<NZ>(&tin, &tout, c, blockIdx.x, smem_raw);
}

template <int NZ, bool SWZ>
__global__ void __launch_bounds__(kT, 2) k_pencil_fast(const C2<float>* in, C2<float>* out, PassCfg c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pencil_item<NZ, SWZ>(in, out, c, blockIdx.x, smem_raw);
}

// ---------------------------------------------------------------- dispatch
namespace {
template <class K, class... Args>
cudaError_t launch_kb(K k, dim3 grid, int nthr, size_t smem, int cluster, cudaStream_t st, Args... args) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(nthr);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (cluster > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, k, args...);
}

template <class K, class... Args>
cudaError_t launch_k(K k, dim3 grid, size_t smem, int cluster, cudaStream_t st, Args... args) {
  return launch_kb(k, grid, kT, smem, cluster, st, args...);
}

// smallest cluster that lets two CTAs share an SM
// clusters of cs CTAs (kT threads, smem bytes each) of kernel k resident at once on the
// device; 0 if the query fails
template <class K>
int resident_clusters(K k, int cs, size_t smem, int nthr = kT) {
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs, 1024);
  cfg.blockDim = dim3(nthr);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  cudaError_t e;
  if (cs > 1) {
    e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
  } else {
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, nthr, smem);
    n *= sms;
  }
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    n = 0;
  }
  return n;
}

template <int H, int NY, int CS>
cudaError_t plane_pair_n(bool inverse, const void* in, void* out, const PassCfg& c, cudaStream_t st, bool prefetch = false,
                         int wide = 0) {
  static_assert(H % CS == 0 && NY % CS == 0, "cluster must split rows and columns evenly");
  const dim3 grid(CS, c.ncomp * c.nz);
  if (inverse) {
    static const int wave = resident_clusters(k_plane_inv_n<H, NY, CS, 0>, CS, ninv_smem<H, NY>(CS));
    const int pf = prefetch ? wave : 0;
    if constexpr (NShape<H, NY>::NTH == 8) {
      if (wide == 2)
        return launch_k(k_plane_inv_n<H, NY, CS, 2>, grid, ninv_smem<H, NY>(CS, 2), CS, st,
                        static_cast<const C2<float>*>(in), static_cast<float*>(out), c, pf);
    }
    if (wide == 1)
      return launch_k(k_plane_inv_n<H, NY, CS, 1>, grid, ninv_smem<H, NY>(CS), CS, st,
                      static_cast<const C2<float>*>(in), static_cast<float*>(out), c, pf);
    return launch_k(k_plane_inv_n<H, NY, CS, 0>, grid, ninv_smem<H, NY>(CS), CS, st,
                    static_cast<const C2<float>*>(in), static_cast<float*>(out), c, pf);
  }
  static const int fwave = resident_clusters(k_plane_fwd_n<H, NY, CS>, CS, nfwd_smem<H, NY>(CS));
  return launch_k(k_plane_fwd_n<H, NY, CS>, grid, nfwd_smem<H, NY>(CS), CS, st, static_cast<const int32_t*>(in),
                  static_cast<C2<float>*>(out), c, wide == 1 ? fwave : 0);
}

// smallest cluster whose CTAs fit two per SM
template <int H, int NY>
__host__ __device__ constexpr bool ncs_fits(int cs) {
  return H % cs == 0 && NY % cs == 0 && nfwd_smem<H, NY>(cs) <= 112 * 1024 && ninv_smem<H, NY>(cs) <= 112 * 1024;
}
template <int H, int NY>
__host__ __device__ constexpr int ncs() {
  return ncs_fits<H, NY>(1) ? 1 : ncs_fits<H, NY>(2) ? 2 : ncs_fits<H, NY>(4) ? 4 : 8;
}

// staged inverse pass: smallest cluster (<= 8) whose CTAs need at most `limit` bytes
template <int H, int NY>
constexpr int stage_cs(size_t limit) {
  for (int cs = 1; cs <= 8; cs *= 2)
    if (H % cs == 0 && NY % cs == 0 && sinv_smem<H, NY>(cs) <= limit) return cs;
  return 0;
}
constexpr size_t kTwoPerSM = 112 * 1024, kThreePerSM = 74 * 1024;

template <int H, int NY, int CS, int NTHR, int MINB>
cudaError_t plane_inv_staged(const void* in, void* out, const PassCfg& c, cudaStream_t st) {
  if constexpr (CS == 0) {
    return cudaErrorInvalidConfiguration;
  } else {
    const dim3 grid(CS, c.ncomp * c.nz);
    return launch_kb(k_plane_inv_s<H, NY, CS, NTHR, MINB>, grid, NTHR, sinv_smem<H, NY>(CS), CS, st,
                     static_cast<const C2<float>*>(in), static_cast<float*>(out), c);
  }
}

// Inverse-pass variants: 0 register-loaded columns (cluster of ncs CTAs, 256 threads);
// staged: 1 with 256 threads and two CTAs per SM, 2 with 128 threads and three CTAs
// per SM, 3 with 256 threads and three CTAs per SM (registers capped at 85); 4 as 0,
// with the next wave's columns prefetched into L2; 5 and 6 as 0 and 4 with the wide
// copy-out of the column outputs; 7 as 6 with 16-byte stores in the copy-out (lines of
// 8 threads, nx >= 128, and only while the wider rows keep two CTAs per SM).
template <int H, int NY>
int plane_inv_variants() {
  constexpr bool w16 = NShape<H, NY>::NTH == 8 && ninv_smem<H, NY>(ncs<H, NY>(), 2) <= kTwoPerSM;
  return 1 | 16 | 32 | 64 | (w16 ? 128 : 0) | (stage_cs<H, NY>(kTwoPerSM) ? 2 : 0) | (stage_cs<H, NY>(kThreePerSM) ? 4 | 8 : 0);
}

template <int H, int NY>
cudaError_t plane_pair(bool inverse, int variant, const void* in, void* out, const PassCfg& c, cudaStream_t st) {
  if (inverse && variant == 1) return plane_inv_staged<H, NY, stage_cs<H, NY>(kTwoPerSM), 256, 2>(in, out, c, st);
  if (inverse && variant == 2) return plane_inv_staged<H, NY, stage_cs<H, NY>(kThreePerSM), 128, 3>(in, out, c, st);
  if (inverse && variant == 3) return plane_inv_staged<H, NY, stage_cs<H, NY>(kThreePerSM), 256, 3>(in, out, c, st);
  if (!inverse) return plane_pair_n<H, NY, ncs<H, NY>()>(false, in, out, c, st, false, variant == 1 ? 1 : 0);
  return plane_pair_n<H, NY, ncs<H, NY>()>(true, in, out, c, st, variant == 4 || variant == 6 || variant == 7,
                                          variant == 7 ? 2 : (variant == 5 || variant == 6) ? 1 : 0);
}

template <int NZ>
cudaError_t pencil_one(int variant, const C2<float>* in, C2<float>* out, const CUtensorMap* tin, const CUtensorMap* tout,
                       const PassCfg& c, cudaStream_t st) {
  const size_t P = (size_t)(c.H + 1) * c.ny;
  const dim3 grid((unsigned)(P / kTW));
  if (variant == 2) {
    if (!tin || !tout) return cudaErrorInvalidValue;
    return launch_k(k_pencil_tma<NZ>, grid, pencil_tma_smem<NZ>(), 1, st, *tin, *tout, c);
  }
  if (variant == 1)
    return launch_k(k_pencil_fast<NZ, false>, grid, pencil_fast_smem<NZ, false>(), 1, st, in, out, c);
  return launch_k(k_pencil_fast<NZ, true>, grid, pencil_fast_smem<NZ, true>(), 1, st, in, out, c);
}

// Pencil variants (one tile per CTA, two CTAs per SM): 0 swizzled tile by 16-byte
// cp.async, 1 padded tile by 8-byte cp.async, 2 swizzled tile by TMA box copies (needs
// the spectra's tensor maps).  A persistent, double-buffered form (one CTA of 384
// threads per SM) measured 1.3-1.6x slower: the transform phase needs the warps more
// than the loads need hiding.
template <int NZ>
int pencil_variants() {
  return 7;
}
}  // namespace

// ---------------------------------------------------------------- batched ensemble passes
// Kernels over work lists of (replica, plane) or (replica, tile) items for an ensemble of
// replicas of uneven edges, one kernel per pass and edge class, with the same bodies,
// cluster sizes and results as the single-grid kernels.  Edges 64, 96, 128, 160, 192 and
// 256 (nx = ny); other grids batch through graphs.
#define OKMC_BATCH_EDGES(X) X(64, 32) X(96, 48) X(128, 64) X(160, 80) X(192, 96) X(256, 128)

template <int H, int NY>
__host__ __device__ constexpr int batch_inv_wide() {
  return NShape<H, NY>::NTH == 8 && ninv_smem<H, NY>(ncs<H, NY>(), 2) <= kTwoPerSM ? 2 : 0;
}

// The pass configurations of batched replicas live in constant memory (slots handed out
// to batches by the host), where the pass bodies read them as they read a kernel
// parameter: immutable, so the compiler keeps or re-reads fields freely, whereas a
// configuration in global memory must be re-read after every store the body makes.
constexpr int kBatchSlots = 128;
__constant__ PassCfg g_batch_cfg[kBatchSlots];

cudaError_t upload_batch_cfg(int slot0, const PassCfg* cfgs, int n, cudaStream_t st) {
  if (slot0 < 0 || n < 0 || slot0 + n > kBatchSlots) return cudaErrorInvalidValue;
  return cudaMemcpyToSymbolAsync(g_batch_cfg, cfgs, n * sizeof(PassCfg), slot0 * sizeof(PassCfg), cudaMemcpyHostToDevice,
                                 st);
}
int batch_cfg_slots() { return kBatchSlots; }

// One work-list kernel per pass and edge class: cluster (plane passes, the edge's own
// cluster size) or CTA (pencil) k runs item k of the list, a plane or tile of any replica
// of that edge.  One item per CTA keeps the bodies at the register count of the
// single-grid kernels (a persistent loop's state pushed them into spills).
template <int H, int NY>
__global__ void __launch_bounds__(kNT, 2) k_fwd_batch(const BatchRep* __restrict__ reps, const int2* __restrict__ items,
                                                      int slot0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 w = items[blockIdx.x / ncs<H, NY>()];
  plane_fwd_item<H, NY, ncs<H, NY>()>(reps[w.x].eps, reps[w.x].spec, g_batch_cfg[slot0 + w.x], w.y, smem_raw);
}

template <int NZ>
__global__ void __launch_bounds__(kT, 2) k_pencil_batch(const BatchRep* __restrict__ reps, const int2* __restrict__ items,
                                                        int slot0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 w = items[blockIdx.x];
  pencil_item<NZ, true>(reps[w.x].spec, reps[w.x].spec2, g_batch_cfg[slot0 + w.x], w.y, smem_raw);
}

template <int H, int NY>
__global__ void __launch_bounds__(kNT, 2) k_inv_batch(const BatchRep* __restrict__ reps, const int2* __restrict__ items,
                                                      int slot0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 w = items[blockIdx.x / ncs<H, NY>()];
  plane_inv_item<H, NY, ncs<H, NY>(), batch_inv_wide<H, NY>()>(reps[w.x].spec2, reps[w.x].sig, g_batch_cfg[slot0 + w.x],
                                                                w.y, 0, 0, smem_raw);
}

bool batch_edge_supported(int nx, int ny, int nz) {
  auto ok = [](int n) { return n == 64 || n == 96 || n == 128 || n == 160 || n == 192 || n == 256; };
  return nx == ny && ok(ny) && ok(nz);
}

// dynamic shared memory of each batched pass for a replica of edge ny (plane passes) / nz
size_t batch_smem(int pass, int n) {
  switch (n) {
#define OKMC_CASE(e, h)                                                          \
  case e:                                                                      \
    return pass == 0 ? nfwd_smem<h, e>(ncs<h, e>())                            \
                     : pass == 1 ? pencil_fast_smem<e, true>()                 \
                                 : ninv_smem<h, e>(ncs<h, e>(), batch_inv_wide<h, e>());
    OKMC_BATCH_EDGES(OKMC_CASE)
#undef OKMC_CASE
    default: return 0;
  }
}

// Grid of a batched pass (0 forward plane, 1 pencil, 2 inverse plane) over nitems items for
// replicas of edge n (one cluster, or CTA, per item); 0 for an edge without batched kernels.
int pass_batch_grid(int pass, int n, int nitems) {
  switch (n) {
#define OKMC_CASE(e, h) \
  case e: return pass == 1 ? nitems : nitems * ncs<h, e>();
    OKMC_BATCH_EDGES(OKMC_CASE)
#undef OKMC_CASE
    default: return 0;
  }
}

// Launch batched pass `pass` for the replicas of edge n over their work list.
cudaError_t launch_pass_batch(int pass, int n, const BatchRep* reps, const int2* items, int nitems, int grid, int slot0,
                              cudaStream_t st) {
  if (nitems == 0) return cudaSuccess;
  switch (n) {
#define OKMC_CASE(e, h)                                                                                            \
  case e:                                                                                                        \
    if (pass == 0)                                                                                               \
      return launch_k(k_fwd_batch<h, e>, dim3(grid), batch_smem(0, e), ncs<h, e>(), st, reps, items, slot0);    \
    if (pass == 1) return launch_k(k_pencil_batch<e>, dim3(grid), batch_smem(1, e), 1, st, reps, items, slot0); \
    return launch_k(k_inv_batch<h, e>, dim3(grid), batch_smem(2, e), ncs<h, e>(), st, reps, items, slot0);
    OKMC_BATCH_EDGES(OKMC_CASE)
#undef OKMC_CASE
    default: return cudaErrorInvalidConfiguration;
  }
}

// The fast path covers nx = ny in {32, 48, 64, 96, 128, 160, 192, 256, 320} and nz
// in the same set.
bool fast_solve_supported(const PassCfg& c) {
  if (c.ncomp != 6 || c.nx != c.ny) return false;
  auto ok = [](int n) {
    return n == 32 || n == 48 || n == 64 || n == 96 || n == 128 || n == 160 || n == 192 || n == 256 || n == 320;
  };
  return ok(c.nx) && ok(c.nz);
}

#define OKMC_FAST_EDGES(X) X(32, 16) X(48, 24) X(64, 32) X(96, 48) X(128, 64) X(160, 80) X(192, 96) X(256, 128) X(320, 160)

cudaError_t launch_plane_fast(bool inverse, int variant, const void* in, void* out, const PassCfg& c, cudaStream_t st) {
  switch (c.ny) {
#define OKMC_CASE(n, h) \
  case n: return plane_pair<h, n>(inverse, variant, in, out, c, st);
    OKMC_FAST_EDGES(OKMC_CASE)
#undef OKMC_CASE
    default: return cudaErrorInvalidConfiguration;
  }
}

// bit v set: forward-pass variant v exists for this grid (0 plain, 1 with the L2
// prefetch of the next wave's dirty planes)
int plane_fwd_variant_mask(const PassCfg&) { return 3; }

// bit v set: inverse-pass variant v exists for this grid
int plane_inv_variant_mask(const PassCfg& c) {
  switch (c.ny) {
#define OKMC_CASE(n, h) \
  case n: return plane_inv_variants<h, n>();
    OKMC_FAST_EDGES(OKMC_CASE)
#undef OKMC_CASE
    default: return 0;
  }
}

cudaError_t launch_pencil_fast(int variant, const C2<float>* in, C2<float>* out, const CUtensorMap* tin,
                               const CUtensorMap* tout, const PassCfg& c, cudaStream_t st) {
  switch (c.nz) {
#define OKMC_CASE(n, h) \
  case n: return pencil_one<n>(variant, in, out, tin, tout, c, st);
    OKMC_FAST_EDGES(OKMC_CASE)
#undef OKMC_CASE
    default: return cudaErrorInvalidConfiguration;
  }
}

int pencil_variant_mask(const PassCfg& c) {
  switch (c.nz) {
#define OKMC_CASE(n, h) \
  case n: return pencil_variants<n>();
    OKMC_FAST_EDGES(OKMC_CASE)
#undef OKMC_CASE
    default: return 0;
  }
}

}  // namespace okmc
