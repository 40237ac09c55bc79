// Dislocation lines as eigenstrain by static field dislocation mechanics (Sec. 2.2:
// Eqs. curlUe, Nye2, eq_EIG_fourier and plastic_0).
//
//   1. k_nye_spread: the Nye tensor alpha_ij(x) = int_L rho_b(x - s) t_j(s) dL_s
//      (Eq. Nye2) of polyline dislocations.  Each segment is cut into m sub-segments of
//      length at most ds_max; the Burgers vector density of a sub-segment, b_i t_j ds / h^3,
//      is spread to the 8 voxel centres around its midpoint with trilinear weights (the
//      core spread over the 8 surrounding grid points, Sec. 4).  Accumulated in int64 fixed
//      point (quantum 2^-40), so the sum does not depend on the order of the atomics.
//   2. the generic forward plane pass transforms the nine components along x and y.
//   3. k_pencil_fdm: per tile of consecutive ky at one kx, the z transform of the nine
//      components, then per frequency the incompatible plastic distortion
//        U_ij = -i xi_k / |xi|^2 eps_jkl alpha_il          (xi != 0, Eq. eq_EIG_fourier)
//      and at xi = 0 the compatible part U(0) = sum over closed lines of
//      (b (x) A + A (x) b) / (2 V) (Eq. plastic_0), then the symmetric part (the plastic
//      strain, taken as eigenstrain) and the inverse z transform of its six components.
//      On a Nyquist plane the operator is averaged over the sign of the Nyquist component,
//      which is what the real part of the inverse of the full spectrum gives: the Nyquist
//      components drop out of the numerator and stay in |xi|^2.
//   4. the generic inverse plane pass; k_quantise_bg rounds the plastic strain to the
//      grid's fixed-point eigenstrain quantum.
//
// A closed line's oriented area A is -1/2 sum_a x_a x x_{a+1}: the line runs clockwise
// seen from the tip of A, so that curl U^p = -alpha holds with U^p = b (x) n on the
// surface the line bounds.
#include "okmc_internal.cuh"

namespace okmc {

template <class T, class Q> cudaError_t launch_plane_fwd(const Q* eps, C2<T>* spec, const PassCfg& c, cudaStream_t st);
template <class T> cudaError_t launch_plane_inv(const C2<T>* spec, T* sig, const PassCfg& c, cudaStream_t st);

namespace {

constexpr int kThreadsFdm = 256;
constexpr int kWarpsFdm = kThreadsFdm / 32;
constexpr double kAlphaQuantum = 9.094947017729282e-13;  // 2^-40
constexpr double kAlphaScale = 1099511627776.0;          // 2^40
constexpr double kAlphaLimit = 4.0e18;                   // |fixed-point value| bound below 2^62

__device__ __forceinline__ int wrap(long long i, int n) {
  long long r = i % n;
  return (int)(r < 0 ? r + n : r);
}

// One block per segment (seg[s] = {first vertex, second vertex} in the flat point array).
__global__ void __launch_bounds__(kThreadsFdm) k_nye_spread(const double* __restrict__ pts, const int2* __restrict__ seg,
                                                            const int* __restrict__ seg_line, const double* __restrict__ burgers,
                                                            int3 n, double h, double ds_max,
                                                            unsigned long long* __restrict__ alpha_q, int* err) {
  const int s = blockIdx.x;
  const int2 ab = seg[s];
  const int l = seg_line[s];
  const double p[3] = {pts[3 * ab.x], pts[3 * ab.x + 1], pts[3 * ab.x + 2]};
  const double d[3] = {__dsub_rn(pts[3 * ab.y], p[0]), __dsub_rn(pts[3 * ab.y + 1], p[1]),
                       __dsub_rn(pts[3 * ab.y + 2], p[2])};
  const double L = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2])));
  if (!(L > 0.0)) return;  // rejected on the host
  const long long m = max(1ll, (long long)ceil(__ddiv_rn(L, ds_max)));
  const double ds = __ddiv_rn(L, (double)m);
  const double t[3] = {__ddiv_rn(d[0], L), __ddiv_rn(d[1], L), __ddiv_rn(d[2], L)};
  const double b[3] = {burgers[3 * l], burgers[3 * l + 1], burgers[3 * l + 2]};
  const double wds = __ddiv_rn(ds, __dmul_rn(__dmul_rn(h, h), h));
  double bt[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) bt[3 * i + j] = __dmul_rn(__dmul_rn(b[i], t[j]), wds);
  const size_t N = (size_t)n.x * n.y * n.z;
  for (long long k = threadIdx.x; k < m; k += blockDim.x) {
    const double off = __dmul_rn((double)k + 0.5, ds);
    double u[3];
    long long i0[3];
    double f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      u[a] = __dsub_rn(__ddiv_rn(__dadd_rn(p[a], __dmul_rn(off, t[a])), h), 0.5);
      const double fl = floor(u[a]);
      i0[a] = (long long)fl;
      f[a] = __dsub_rn(u[a], fl);
    }
    const int ix[2] = {wrap(i0[0], n.x), wrap(i0[0] + 1, n.x)};
    const int iy[2] = {wrap(i0[1], n.y), wrap(i0[1] + 1, n.y)};
    const int iz[2] = {wrap(i0[2], n.z), wrap(i0[2] + 1, n.z)};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int cx = (c >> 2) & 1, cy = (c >> 1) & 1, cz = c & 1;
      const double w = __dmul_rn(__dmul_rn(cx ? f[0] : __dsub_rn(1.0, f[0]), cy ? f[1] : __dsub_rn(1.0, f[1])),
                                 cz ? f[2] : __dsub_rn(1.0, f[2]));
      const size_t v = ((size_t)iz[cz] * n.y + iy[cy]) * n.x + ix[cx];
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const double val = __dmul_rn(__dmul_rn(w, bt[q]), kAlphaScale);
        if (!(fabs(val) < kAlphaLimit)) {
          atomicExch(err, 4);
          continue;
        }
        atomicAdd(alpha_q + q * N + v, (unsigned long long)llrint(val));
      }
    }
  }
}

// Oriented area of each closed line, A = -1/2 sum_a x_a x x_{a+1} (one block per line;
// per-thread partial sums over a fixed stride, then a fixed-order reduction).
__global__ void __launch_bounds__(kThreadsFdm) k_line_area(const double* __restrict__ pts, const int* __restrict__ first,
                                                           const int* __restrict__ closed, double* __restrict__ area) {
  __shared__ double sh[3][kThreadsFdm];
  const int l = blockIdx.x;
  const int a0 = first[l], a1 = first[l + 1];
  double acc[3] = {0.0, 0.0, 0.0};
  if (closed[l]) {
    for (int a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
      const int b = a + 1 < a1 ? a + 1 : a0;
      const double* x = pts + 3 * a;
      const double* y = pts + 3 * b;
      acc[0] += __dsub_rn(__dmul_rn(x[1], y[2]), __dmul_rn(x[2], y[1]));
      acc[1] += __dsub_rn(__dmul_rn(x[2], y[0]), __dmul_rn(x[0], y[2]));
      acc[2] += __dsub_rn(__dmul_rn(x[0], y[1]), __dmul_rn(x[1], y[0]));
    }
  }
  for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) area[3 * l + threadIdx.x] = -0.5 * sh[threadIdx.x][0];
}

struct FdmArgs {
  const double* burgers;  // [nl][3]
  const double* area;     // [nl][3] (zero for open lines)
  int nl;
  double h;
  double volume;          // box volume nx ny nz h^3
};

template <class T>
__host__ __device__ inline size_t pencil_fdm_smem(int nz, int tw) {
  return sizeof(C2<T>) * ((size_t)9 * tw * (nz + 1) + nz + (size_t)kWarpsFdm * 2 * nz);
}

// In place on the spectrum: reads the nine transformed Nye-tensor components of its
// tile, writes the six plastic-strain components (component slots 0..5).
template <class T>
__global__ void __launch_bounds__(kThreadsFdm) k_pencil_fdm(C2<T>* __restrict__ spec, PassCfg c, int TW, FdmArgs f) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nz = c.nz, ldl = nz + 1;
  C2<T>* lines = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* twZ = lines + (size_t)9 * TW * ldl;
  C2<T>* scr = twZ + nz;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t P = (size_t)(c.H + 1) * c.ny;
  const size_t p0 = (size_t)blockIdx.x * TW;
  const int kx = (int)(p0 / c.ny), ky0 = (int)(p0 % c.ny);
  const C2<T>* gZ = reinterpret_cast<const C2<T>*>(c.twZ);
  for (int i = threadIdx.x; i < nz; i += blockDim.x) twZ[i] = gZ[i];
  const int total9 = 9 * nz * TW;
  for (int idx = threadIdx.x; idx < total9; idx += blockDim.x) {
    const int t = idx % TW, kz = (idx / TW) % nz, comp = idx / (TW * nz);
    lines[(size_t)(comp * TW + t) * ldl + kz] = spec[((size_t)comp * nz + kz) * P + p0 + t];
  }
  __syncthreads();
  C2<T>* bufA = scr + (size_t)warp * 2 * nz;
  C2<T>* bufB = bufA + nz;
  for (int l = warp; l < 9 * TW; l += kWarpsFdm) {
    SLine<T> ln{lines + (size_t)l * ldl, 1};
    line_fft<T, false>(ln, ln, bufA, bufB, twZ, c.pZ, lane);
  }
  __syncthreads();
  const double rN = 1.0 / ((double)c.nx * (double)c.ny * (double)c.nz);
  for (int idx = threadIdx.x; idx < TW * nz; idx += blockDim.x) {
    const int t = idx / nz, kz = idx % nz;
    const int ky = ky0 + t;
    const int fx = kx < c.H ? kx : kx - c.nx;
    const int fy = ky < c.ny / 2 ? ky : ky - c.ny;
    const int fz = kz < c.nz / 2 ? kz : kz - c.nz;
    C2<T> e6[6];
    if (fx == 0 && fy == 0 && fz == 0) {
      double U[3][3] = {};
      for (int l = 0; l < f.nl; ++l)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            U[i][j] += (f.burgers[3 * l + i] * f.area[3 * l + j] + f.area[3 * l + i] * f.burgers[3 * l + j]) / (2.0 * f.volume);
      const double v6[6] = {U[0][0], U[1][1], U[2][2], 0.5 * (U[1][2] + U[2][1]), 0.5 * (U[0][2] + U[2][0]),
                            0.5 * (U[0][1] + U[1][0])};
      for (int a = 0; a < 6; ++a) e6[a] = C2<T>{(T)v6[a], T(0)};
    } else {
      const double q[3] = {(double)fx / c.nx, (double)fy / c.ny, (double)fz / c.nz};
      const double q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
      // xi_k / |xi|^2 = h q_k / (2 pi |q|^2), times 1/N for the unnormalised inverse
      const double s = f.h / (2.0 * kPi * q2) * rN;
      const T g[3] = {(T)((kx == c.H ? 0.0 : q[0]) * s), (T)((2 * ky == c.ny ? 0.0 : q[1]) * s),
                      (T)((2 * kz == c.nz ? 0.0 : q[2]) * s)};
      C2<T> U[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        C2<T> a[3];
#pragma unroll
        for (int l = 0; l < 3; ++l) a[l] = lines[(size_t)((3 * i + l) * TW + t) * ldl + kz];
        // (g x a)_j = eps_jkl g_k a_l; U_ij = -i (g x a)_j
        const C2<T> cr[3] = {g[1] * a[2] - g[2] * a[1], g[2] * a[0] - g[0] * a[2], g[0] * a[1] - g[1] * a[0]};
#pragma unroll
        for (int j = 0; j < 3; ++j) U[i][j] = C2<T>{cr[j].y, -cr[j].x};
      }
      e6[0] = U[0][0];
      e6[1] = U[1][1];
      e6[2] = U[2][2];
      e6[3] = T(0.5) * (U[1][2] + U[2][1]);
      e6[4] = T(0.5) * (U[0][2] + U[2][0]);
      e6[5] = T(0.5) * (U[0][1] + U[1][0]);
    }
    // only this thread reads or writes point (t, kz): slots 0..5 can be overwritten in place
    for (int a = 0; a < 6; ++a) lines[(size_t)(a * TW + t) * ldl + kz] = e6[a];
  }
  __syncthreads();
  for (int l = warp; l < 6 * TW; l += kWarpsFdm) {
    SLine<T> ln{lines + (size_t)l * ldl, 1};
    line_fft<T, true>(ln, ln, bufA, bufB, twZ, c.pZ, lane);
  }
  __syncthreads();
  const int total6 = 6 * nz * TW;
  for (int idx = threadIdx.x; idx < total6; idx += blockDim.x) {
    const int t = idx % TW, kz = (idx / TW) % nz, comp = idx / (TW * nz);
    spec[((size_t)comp * nz + kz) * P + p0 + t] = lines[(size_t)(comp * TW + t) * ldl + kz];
  }
}

template <class T, class Q>
__global__ void k_quantise_bg(const T* __restrict__ u, Q* __restrict__ out, size_t count, double rq, double lim, int* err) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const double v = (double)u[i] * rq;
    if (!(fabs(v) <= lim)) {
      atomicExch(err, 4);
      out[i] = 0;
      continue;
    }
    out[i] = (Q)llrint(v);
  }
}

}  // namespace

template <class T>
int fdm_pencil_tile(int ny, int nz, size_t limit) {
  for (int tw = 8; tw >= 1; tw /= 2) {
    if (ny % tw) continue;
    if (pencil_fdm_smem<T>(nz, tw) <= limit) return tw;
  }
  return 0;
}
template int fdm_pencil_tile<float>(int, int, size_t);
template int fdm_pencil_tile<double>(int, int, size_t);

// Device side of okmc_set_dislocations.  alpha_q: 9 N int64 (zeroed here); spec: 9 nz P
// complex T; bg: 6 N Q.  The plastic strain in T passes through alpha_q's memory once the
// forward pass has consumed it.  Returns the first failing CUDA call's error.
template <class T, class Q>
cudaError_t launch_dislocation_eigenstrain(const double* pts, const int2* seg, const int* seg_line, int nseg,
                                           const int* first, const int* closed, const double* burgers, double* area,
                                           int nl, double ds_max, const PassCfg& c0, double h, int tw,
                                           unsigned long long* alpha_q, C2<T>* spec, Q* bg, double q, double qlim,
                                           int* err, cudaStream_t st) {
  const int3 n = make_int3(c0.nx, c0.ny, c0.nz);
  const size_t N = (size_t)n.x * n.y * n.z;
  cudaError_t e = cudaMemsetAsync(alpha_q, 0, 9 * N * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (nseg > 0) {
    k_nye_spread<<<nseg, kThreadsFdm, 0, st>>>(pts, seg, seg_line, burgers, n, h, ds_max, alpha_q, err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_line_area<<<nl, kThreadsFdm, 0, st>>>(pts, first, closed, area);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  PassCfg c = c0;
  c.ncomp = 9;
  c.q = kAlphaQuantum;
  c.forward_only = 0;
  c.dirty = nullptr;
  e = launch_plane_fwd<T, int64_t>(reinterpret_cast<const int64_t*>(alpha_q), spec, c, st);
  if (e != cudaSuccess) return e;
  const size_t smem = pencil_fdm_smem<T>(c.nz, tw);
  e = cudaFuncSetAttribute(k_pencil_fdm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const size_t P = (size_t)(c.H + 1) * c.ny;
  FdmArgs f{burgers, area, nl, h, (double)N * h * h * h};
  k_pencil_fdm<T><<<(unsigned)(P / tw), kThreadsFdm, smem, st>>>(spec, c, tw, f);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  c.ncomp = 6;
  T* u = reinterpret_cast<T*>(alpha_q);
  e = launch_plane_inv<T>(spec, u, c, st);
  if (e != cudaSuccess) return e;
  k_quantise_bg<T, Q><<<1024, 256, 0, st>>>(u, bg, 6 * N, 1.0 / q, qlim, err);
  return cudaGetLastError();
}

template cudaError_t launch_dislocation_eigenstrain<float, int32_t>(const double*, const int2*, const int*, int, const int*,
                                                                    const int*, const double*, double*, int, double,
                                                                    const PassCfg&, double, int, unsigned long long*,
                                                                    C2<float>*, int32_t*, double, double, int*, cudaStream_t);
template cudaError_t launch_dislocation_eigenstrain<double, int64_t>(const double*, const int2*, const int*, int, const int*,
                                                                     const int*, const double*, double*, int, double,
                                                                     const PassCfg&, double, int, unsigned long long*,
                                                                     C2<double>*, int64_t*, double, double, int*,
                                                                     cudaStream_t);

}  // namespace okmc
