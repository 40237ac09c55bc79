// The paper's own evaluation of a defect's interaction energy at continuous positions
// (Sec. 3.3, Eq. shift; Sec. 2 Eq. interaction_energy3 in its elastic-strain form):
//
//   E_i(X) = kappa int sigma^(-i) : eps^e_i(. - X) dV
//          = kappa (h^3 / N) Re sum_xi conj(sigma^(-i)_hat(xi)) : eps^e_ref_hat(xi) exp(-i xi.X)
//
// eps^e_ref is the elastic strain C^-1 : sigma_ref of defect i alone with its class-0
// stencil placed at the origin (its centre at X0 = 0), moved to X by the phase factor of
// the shift theorem and summed by Parseval over the discrete frequencies of Sec. 3.4.
// sigma^(-i) is the stress of everything on the grid except defect i at its current site.
//
// Both spectra come from the Green operator per frequency:
//   sigma^(-i)_hat = G(eps*_hat - alpha_c e W_c(xi) exp(-i xi.b h)),
//   sigma_ref_hat  = G(alpha_0 e W_0(xi)),
// with eps*_hat the transformed eigenstrain of the grid, W_c the transformed count field
// of defect i's class-c stencil at the origin and b its current base voxel.  On the
// stored half spectrum the full sum is, per stored frequency: the kx = 0 and kx = nx/2
// planes once with their own phase; 0 < kx < nx/2 twice, with the phase averaged over the
// sign of the y and z Nyquist components (flipped together), which is the mirror
// frequency's contribution under the Hermitian symmetry of both spectra.
#include "okmc_internal.cuh"

namespace okmc {

constexpr int kShiftMax = 8;  // positions per pass over the spectrum

namespace {

constexpr int kShiftThreads = 256;

__device__ __forceinline__ double shift_block_sum(double v, double* sh) {
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

template <class T>
__device__ __forceinline__ C2<T> scale_c(T s, C2<T> a) {
  return C2<T>{s * a.x, s * a.y};
}

// One block-stride pass over the half spectrum for up to kShiftMax positions.
template <class T>
__global__ void __launch_bounds__(kShiftThreads) k_shift_partial(const C2<T>* __restrict__ spec_e,
                                                                 const C2<T>* __restrict__ spec_w, PassCfg c,
                                                                 const okmc_defect* __restrict__ def,
                                                                 const DefGeo* __restrict__ G,
                                                                 const double* __restrict__ alpha, int i,
                                                                 const double* __restrict__ X, int m, double h,
                                                                 double* __restrict__ partial) {
  __shared__ double sh[32];
  const size_t P = (size_t)(c.H + 1) * c.ny;
  const size_t total = P * c.nz;
  const int pos[3] = {def[i].pos[0], def[i].pos[1], def[i].pos[2]};
  const int cls = pos[0] & 1;
  const int b[3] = {floor_div2(pos[0]), floor_div2(pos[1]), floor_div2(pos[2])};
  const DefGeo g = G[i];
  const T a0 = (T)alpha[2 * i], ac = (T)alpha[2 * i + cls];
  const double C11 = c.C11, C12 = c.C12, C44 = c.C44;
  const double den = (C11 - C12) * (C11 + 2.0 * C12);
  const double S11 = (C11 + C12) / den, S12 = -C12 / den, S44h = 0.5 / C44;  // tensor shear strain = s / (2 C44)
  double xs[kShiftMax][3];
  double acc[kShiftMax];
#pragma unroll
  for (int k = 0; k < kShiftMax; ++k) {
    acc[k] = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) xs[k][a] = k < m ? X[3 * k + a] / h : 0.0;  // positions in voxels
  }
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int kz = (int)(idx / P);
    const int p = (int)(idx % P);
    const int kx = p / c.ny, ky = p % c.ny;
    const C2<T> w0 = spec_w[(size_t)kz * P + p];
    const C2<T> wc = spec_w[((size_t)cls * c.nz + kz) * P + p];
    // exp(-2 pi i k.b / n) for the current base voxel (integer phases reduced exactly)
    const double fb = (double)(((long long)kx * b[0]) % c.nx) / c.nx + (double)(((long long)ky * b[1]) % c.ny) / c.ny +
                      (double)(((long long)kz * b[2]) % c.nz) / c.nz;
    double sb, cb;
    sincospi(2.0 * fb, &sb, &cb);
    const C2<T> wcb{(T)((double)wc.x * cb + (double)wc.y * sb), (T)((double)wc.y * cb - (double)wc.x * sb)};
    C2<T> ex[6], er[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      const C2<T> e = spec_e[((size_t)a * c.nz + kz) * P + p];
      const T ea = (T)g.e6[a];
      ex[a] = e - scale_c(ac * ea, wcb);
      er[a] = scale_c(a0 * ea, w0);
    }
    green_point<T>(ex, kx, ky, kz, c, T(1));  // sigma^(-i)_hat
    green_point<T>(er, kx, ky, kz, c, T(1));  // sigma_ref_hat
    // eps^e_ref = C^-1 : sigma_ref (tensor components), then A = conj(sigma^(-i)) : eps^e_ref
    double Ar = 0.0, Ai = 0.0;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      double erx, ery;
      if (a < 3) {
        const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
        erx = S11 * er[a].x + S12 * ((double)er[a1].x + er[a2].x);
        ery = S11 * er[a].y + S12 * ((double)er[a1].y + er[a2].y);
      } else {
        erx = 2.0 * S44h * er[a].x;  // factor 2: the off-diagonal pair of a : b
        ery = 2.0 * S44h * er[a].y;
      }
      Ar += (double)ex[a].x * erx + (double)ex[a].y * ery;
      Ai += (double)ex[a].x * ery - (double)ex[a].y * erx;
    }
    const int fx = kx < c.H ? kx : kx - c.nx;
    const int fy = ky < c.ny / 2 ? ky : ky - c.ny;
    const int fz = kz < c.nz / 2 ? kz : kz - c.nz;
    const bool inner = kx > 0 && kx < c.H;
    const bool flip = inner && (2 * ky == c.ny || 2 * kz == c.nz);
    const int fy2 = (2 * ky == c.ny) ? -fy : fy, fz2 = (2 * kz == c.nz) ? -fz : fz;
#pragma unroll
    for (int k = 0; k < kShiftMax; ++k) {
      if (k >= m) break;
      // Re(A exp(-i theta)) = Ar cos(theta) + Ai sin(theta), theta = 2 pi sum_a f_a x_a / n_a
      double s, co;
      sincospi(2.0 * ((double)fx * xs[k][0] / c.nx + (double)fy * xs[k][1] / c.ny + (double)fz * xs[k][2] / c.nz), &s, &co);
      double v = Ar * co + Ai * s;
      if (flip) {
        double s2, co2;
        sincospi(2.0 * ((double)fx * xs[k][0] / c.nx + (double)fy2 * xs[k][1] / c.ny + (double)fz2 * xs[k][2] / c.nz),
                 &s2, &co2);
        v = 0.5 * (v + Ar * co2 + Ai * s2);
      }
      acc[k] += inner ? 2.0 * v : v;
    }
  }
#pragma unroll
  for (int k = 0; k < kShiftMax; ++k) {
    if (k >= m) break;  // m is uniform over the block: every thread takes the same path
    const double t = shift_block_sum(acc[k], sh);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * kShiftMax + k] = t;
  }
}

__global__ void k_shift_final(const double* __restrict__ partial, int nblocks, int m, double scale, double* __restrict__ E) {
  const int k = threadIdx.x;
  if (k >= m) return;
  double t = 0.0;
  for (int bl = 0; bl < nblocks; ++bl) t += partial[(size_t)bl * kShiftMax + k];
  E[k] = scale * t;
}

}  // namespace

int shift_positions_per_pass() { return kShiftMax; }

// partial: nblocks * kShiftMax doubles.  X: m <= kShiftMax positions (nm, device).
template <class T>
cudaError_t launch_shift_energies(const C2<T>* spec_e, const C2<T>* spec_w, const PassCfg& c, const okmc_defect* def,
                                  const DefGeo* G, const double* alpha, int i, const double* X, int m, double h,
                                  double* partial, int nblocks, double* E, cudaStream_t st) {
  if (m <= 0 || m > kShiftMax) return cudaErrorInvalidValue;
  k_shift_partial<T><<<nblocks, kShiftThreads, 0, st>>>(spec_e, spec_w, c, def, G, alpha, i, X, m, h, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const double N = (double)c.nx * c.ny * c.nz;
  k_shift_final<<<1, 32, 0, st>>>(partial, nblocks, m, kKappa * h * h * h / N, E);
  return cudaGetLastError();
}

template cudaError_t launch_shift_energies<float>(const C2<float>*, const C2<float>*, const PassCfg&, const okmc_defect*,
                                                  const DefGeo*, const double*, int, const double*, int, double, double*,
                                                  int, double*, cudaStream_t);
template cudaError_t launch_shift_energies<double>(const C2<double>*, const C2<double>*, const PassCfg&, const okmc_defect*,
                                                   const DefGeo*, const double*, int, const double*, int, double, double*,
                                                   int, double*, cudaStream_t);

}  // namespace okmc
