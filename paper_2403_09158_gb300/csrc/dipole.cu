// Dipole approximation of the interaction energy (Sec. 2.1, Eqs. interaction_energy4,
// dipole_def, dipole_def2; Appendix B).  With the external field taken constant over a
// defect, E_i(Y) ~ -P_i : eps_ext(Y) = -(int eps*_i) : sigma^(-i)(Y), where
// P_i = C : int eps*_i and sigma^(-i) = sigma - sigma_i is the stress of all the other
// defects.  sigma(Y) is read at the centre of a site: the base voxel of a class-1 site
// (its centre), the mean of the 8 voxels around the corner of a class-0 site.  The self
// part
//   D_i(c, k) = (int eps*_i) : sigma_i^c(Y_k),
// the defect's own field at the centre of its site (k = 0) or of its jump k - 1 when it
// sits on a class-c site, is translation invariant and is summed in Fourier space per
// distinct shape, beside the self-term table W:
//   D(c, k) = V_shape a_c s^2 / N  Re sum_xi Q_t(xi) w_c(xi) S_k(xi),
// with w_c the transformed count field of the class-c stencil (base voxel at the
// origin), Q_t the type's stress-energy table and S_k(xi) the mean of exp(+i xi.v) over
// the centre voxels v of Y_k.
#include "okmc_internal.cuh"

namespace okmc {

namespace {

__device__ __forceinline__ double dip_block_sum(double v, double* sh) {
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

// compensated FP32 pairs for FP32 spectra, plain FP64 for FP64 spectra
template <class T> struct DAcc;
template <> struct DAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <> struct DAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};

template <class T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return C2<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// The 18 sums of one shape (defect d of the batch) over the half spectrum (weight 2 off
// the kx = 0 and kx = nx/2 planes).  Per axis, with e = exp(+i xi) (one voxel):
//   class 0, site:      the centre is the corner of voxels {-1, 0}: factor (1 + conj e)/2;
//   class 0, jump j:    the centre is the voxel d = 0 (bit of j set) or -1: 1 or conj e;
//   class 1, site:      the base voxel: 1;
//   class 1, jump j:    the corner of voxels {0, 1} (bit set) or {-1, 0}: (1 + e)/2 or
//                       (1 + conj e)/2.
template <class T, class QT>
__global__ void __launch_bounds__(256) k_dipself_partial(const C2<T>* __restrict__ spec, PassCfg c, WBatch b, int d,
                                                         const QT* __restrict__ qtab, const double2* __restrict__ phx,
                                                         const double2* __restrict__ phy, const double2* __restrict__ phz,
                                                         double* __restrict__ partial) {
  __shared__ double sh[32];
  const size_t P = (size_t)(c.H + 1) * c.ny;
  const size_t total = P * c.nz;
  DAcc<T> acc[18];
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int kz = (int)(idx / P);
    const int p = (int)(idx % P);
    const int kx = p / c.ny, ky = p % c.ny;
    const T wgt = (kx == 0 || kx == c.H) ? T(1) : T(2);
    const double2 ex = phx[kx], ey = phy[ky], ez = phz[kz];
    const C2<T> e[3] = {C2<T>{(T)ex.x, (T)ex.y}, C2<T>{(T)ey.x, (T)ey.y}, C2<T>{(T)ez.x, (T)ez.y}};
    C2<T> lo[3], hi[3], cj[3];  // (1 + conj e)/2, (1 + e)/2, conj e
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = C2<T>{T(0.5) * (T(1) + e[a].x), T(-0.5) * e[a].y};
      hi[a] = C2<T>{T(0.5) * (T(1) + e[a].x), T(0.5) * e[a].y};
      cj[a] = C2<T>{e[a].x, -e[a].y};
    }
    const C2<T> w0 = spec[((size_t)(2 * d) * c.nz + kz) * P + p];
    const C2<T> w1 = spec[((size_t)(2 * d + 1) * c.nz + kz) * P + p];
    const T q = wgt * (T)qtab[(size_t)b.type[d] * total + idx];
    const C2<T> u0{q * w0.x, q * w0.y}, u1{q * w1.x, q * w1.y};
    acc[0].add(cmul(u0, cmul(cmul(lo[0], lo[1]), lo[2])).x);
    acc[9].add(u1.x);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const bool bx = (j >> 2) & 1, by = (j >> 1) & 1, bz = j & 1;
      C2<T> f0{T(1), T(0)};
      if (!bx) f0 = cj[0];
      if (!by) f0 = cmul(f0, cj[1]);
      if (!bz) f0 = cmul(f0, cj[2]);
      const C2<T> f1 = cmul(cmul(bx ? hi[0] : lo[0], by ? hi[1] : lo[1]), bz ? hi[2] : lo[2]);
      acc[1 + j].add(cmul(u0, f0).x);
      acc[10 + j].add(cmul(u1, f1).x);
    }
  }
#pragma unroll
  for (int k = 0; k < 18; ++k) {
    const double t = dip_block_sum(acc[k].value(), sh);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * 18 + k] = t;
  }
}

// D[i][c][k] = (h^3 / N) s^2 (V_shape / h^3) a_c S[c][k] for the batch's defect d.
__global__ void k_dipself_final(const double* __restrict__ partial, int nblocks, WBatch b, int d,
                                const double* __restrict__ alpha, const DefGeo* __restrict__ G, double scale,
                                double* __restrict__ D) {
  const int k = threadIdx.x;
  if (k >= 18) return;
  double t = 0.0;
  for (int bl = 0; bl < nblocks; ++bl) t += partial[(size_t)bl * 18 + k];
  const int i = b.idx[d], cls = k / 9;
  D[(size_t)i * 18 + k] = scale * b.s2[d] * G[i].v_over_h3 * alpha[2 * i + cls] * t;
}

// sigma (6 components) at the centre of a site at half-lattice position p, in FP64
template <class T>
__device__ void centre_stress(const T* __restrict__ sig, int3 n, size_t N, const int p[3], double s[6]) {
  const int bx = floor_div2(p[0]), by = floor_div2(p[1]), bz = floor_div2(p[2]);
  for (int a = 0; a < 6; ++a) s[a] = 0.0;
  if (p[0] & 1) {
    const size_t v = ((size_t)bz * n.y + by) * n.x + bx;
    for (int a = 0; a < 6; ++a) s[a] = (double)sig[a * N + v];
    return;
  }
  for (int m = 0; m < 8; ++m) {  // voxels base + {-1, 0}^3, in a fixed order
    const int x = bx - ((m >> 2) & 1), y = by - ((m >> 1) & 1), z = bz - (m & 1);
    const size_t v = ((size_t)(z < 0 ? z + n.z : z) * n.y + (y < 0 ? y + n.y : y)) * n.x + (x < 0 ? x + n.x : x);
    for (int a = 0; a < 6; ++a) s[a] += (double)sig[a * N + v];
  }
  for (int a = 0; a < 6; ++a) s[a] *= 0.125;
}

// One thread per (defect, position): k = 0 the site, k = 1 + j jump j.
//   E = -kappa (h^3 V_shape/h^3 e : sigma(Y) - D[i][c][k])
template <class T>
__global__ void k_dipole_energies(const T* __restrict__ sig, int3 n, const okmc_defect* __restrict__ def,
                                  const DefGeo* __restrict__ G, const double* __restrict__ D, int nd, double h3,
                                  double* __restrict__ E, double* __restrict__ Ec) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 9 * nd) return;
  const int i = t / 9, k = t % 9;
  const okmc_defect r = def[i];
  const int c = r.pos[0] & 1;
  int p[3] = {r.pos[0], r.pos[1], r.pos[2]};
  if (k > 0) {  // lambda_j = (a0/2)(sx, sy, sz), bit 2: sx > 0, bit 1: sy > 0, bit 0: sz > 0
    const int j = k - 1;
    const int L[3] = {2 * n.x, 2 * n.y, 2 * n.z};
    const int sgn[3] = {(j >> 2) & 1 ? 1 : -1, (j >> 1) & 1 ? 1 : -1, j & 1 ? 1 : -1};
    for (int a = 0; a < 3; ++a) {
      p[a] += sgn[a];
      if (p[a] < 0) p[a] += L[a];
      if (p[a] >= L[a]) p[a] -= L[a];
    }
  }
  double s[6];
  centre_stress<T>(sig, n, (size_t)n.x * n.y * n.z, p, s);
  const DefGeo g = G[i];
  double es = 0.0;
  for (int a = 0; a < 6; ++a) es += (a < 3 ? 1.0 : 2.0) * g.e6[a] * s[a];
  const double e = -kKappa * (h3 * g.v_over_h3 * es - D[(size_t)i * 18 + c * 9 + k]);
  if (k == 0) E[i] = e;
  else if (Ec) Ec[(size_t)i * 8 + k - 1] = e;
}

// Point defects of given dipole tensor P (eV, (xx, yy, zz, yz, xz, xy)) at bcc sites:
// E = -P : eps(Y), eps = C^-1 : sigma at the centre of the site.  For cubic C the
// compliance gives the engineering strains e_a = S11 s_a + S12 (s_b + s_c) (a, b, c the
// three normal components) and gamma = s / C44 (shear), and P : eps = sum_a P_a e_a.
// A site off the lattice or outside the box gives NaN and error code 8.
template <class T>
__global__ void k_point_dipole(const T* __restrict__ sig, int3 n, const int* __restrict__ pos,
                               const double* __restrict__ P, int m, double C11, double C12, double C44,
                               double* __restrict__ E, int* err) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const int p[3] = {pos[3 * k], pos[3 * k + 1], pos[3 * k + 2]};
  const bool inside = p[0] >= 0 && p[1] >= 0 && p[2] >= 0 && p[0] < 2 * n.x && p[1] < 2 * n.y && p[2] < 2 * n.z;
  if (!inside || ((p[0] ^ p[1]) & 1) || ((p[0] ^ p[2]) & 1)) {
    E[k] = nan("");
    atomicExch(err, 8);
    return;
  }
  double s[6];
  centre_stress<T>(sig, n, (size_t)n.x * n.y * n.z, p, s);
  const double den = (C11 - C12) * (C11 + 2.0 * C12);
  const double S11 = (C11 + C12) / den, S12 = -C12 / den;
  const double e[6] = {S11 * s[0] + S12 * (s[1] + s[2]), S11 * s[1] + S12 * (s[0] + s[2]),
                       S11 * s[2] + S12 * (s[0] + s[1]), s[3] / C44, s[4] / C44, s[5] / C44};
  double pe = 0.0;
  for (int a = 0; a < 6; ++a) pe += P[6 * (size_t)k + a] * e[a];
  E[k] = -pe;
}

}  // namespace

template <class T>
cudaError_t launch_point_dipole(const T* sig, int3 n, const int* pos, const double* P, int m, double C11, double C12,
                                double C44, double* E, int* err, cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  k_point_dipole<T><<<(m + 255) / 256, 256, 0, st>>>(sig, n, pos, P, m, C11, C12, C44, E, err);
  return cudaGetLastError();
}
template cudaError_t launch_point_dipole<float>(const float*, int3, const int*, const double*, int, double, double, double,
                                                double*, int*, cudaStream_t);
template cudaError_t launch_point_dipole<double>(const double*, int3, const int*, const double*, int, double, double,
                                                 double, double*, int*, cudaStream_t);

template <class T, class QT>
cudaError_t launch_dipself(const C2<T>* spec, const PassCfg& c, const WBatch& b, const QT* qtab, const double2* phx,
                           const double2* phy, const double2* phz, double* partial, int nblocks, const double* alpha,
                           const DefGeo* G, double scale, double* D, cudaStream_t st) {
  for (int d = 0; d < b.nb; ++d) {
    k_dipself_partial<T, QT><<<nblocks, 256, 0, st>>>(spec, c, b, d, qtab, phx, phy, phz, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_dipself_final<<<1, 32, 0, st>>>(partial, nblocks, b, d, alpha, G, scale, D);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <class T>
cudaError_t launch_dipole_energies(const T* sig, int3 n, const okmc_defect* def, const DefGeo* G, const double* D, int nd,
                                   double h3, double* E, double* Ec, cudaStream_t st) {
  if (nd == 0) return cudaSuccess;
  const int threads = 9 * nd;
  k_dipole_energies<T><<<(threads + 255) / 256, 256, 0, st>>>(sig, n, def, G, D, nd, h3, E, Ec);
  return cudaGetLastError();
}

template cudaError_t launch_dipself<float, float>(const C2<float>*, const PassCfg&, const WBatch&, const float*,
                                                  const double2*, const double2*, const double2*, double*, int,
                                                  const double*, const DefGeo*, double, double*, cudaStream_t);
template cudaError_t launch_dipself<double, double>(const C2<double>*, const PassCfg&, const WBatch&, const double*,
                                                    const double2*, const double2*, const double2*, double*, int,
                                                    const double*, const DefGeo*, double, double*, cudaStream_t);
template cudaError_t launch_dipole_energies<float>(const float*, int3, const okmc_defect*, const DefGeo*, const double*, int,
                                                   double, double*, double*, cudaStream_t);
template cudaError_t launch_dipole_energies<double>(const double*, int3, const okmc_defect*, const DefGeo*, const double*,
                                                    int, double, double*, double*, cudaStream_t);

}  // namespace okmc
