// Internal declarations of the GB300 OkMC elastic-interaction library.
//
// Data layout in device memory (one handle, one grid of nx*ny*nz voxels, x fastest):
//   eps   : eigenstrain, 6 components [c][z][y][x], fixed point (int32 with
//           quantum 2^-26 for FP32 fields, int64 with quantum 2^-40 for FP64
//           fields) so that incremental add/subtract of stencils is exact.
//   sigma : stress, 6 components [c][z][y][x] in T (float or double).
//   spec  : half spectrum, 6 components, per component nz planes of
//           P = (nx/2 + 1) * ny complex values in kx-major order p = kx*ny + ky
//           ("transposed plane"): the forward plane pass writes whole kx columns,
//           the pencil pass reads TW consecutive ky at one kx for every kz.
#pragma once

#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>
#include <stdint.h>

#include "okmc.h"

namespace okmc {

constexpr double kPi = 3.141592653589793;
constexpr double kKappa = 6.241509074;      // eV per GPa nm^3
constexpr double kBoltzmann = 8.617333262e-5;  // eV/K

// ---------------------------------------------------------------- complex
template <class T>
struct alignas(2 * sizeof(T)) C2 {
  T x, y;
};

template <class T> __host__ __device__ __forceinline__ C2<T> operator+(C2<T> a, C2<T> b) { return {a.x + b.x, a.y + b.y}; }
template <class T> __host__ __device__ __forceinline__ C2<T> operator-(C2<T> a, C2<T> b) { return {a.x - b.x, a.y - b.y}; }
template <class T> __host__ __device__ __forceinline__ C2<T> operator*(C2<T> a, C2<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class T> __host__ __device__ __forceinline__ C2<T> operator*(T s, C2<T> a) { return {s * a.x, s * a.y}; }
template <class T> __host__ __device__ __forceinline__ C2<T> conjg(C2<T> a) { return {a.x, -a.y}; }
// multiply by -i (forward transform) or +i (inverse transform)
template <class T, bool INV> __device__ __forceinline__ C2<T> rot(C2<T> v) {
  return INV ? C2<T>{-v.y, v.x} : C2<T>{v.y, -v.x};
}

// ---------------------------------------------------------------- packed FP32 pairs
// The sm_100 family executes add, multiply and fma on a pair of FP32 values in one
// instruction (round to nearest, each lane exactly as the scalar operation), so a
// complex add, subtract or real scaling costs one instruction instead of two.  A
// multiplication by -i or +i swaps the lanes; such terms are added in scalar form.
__device__ __forceinline__ float2 pk(C2<float> a) { return make_float2(a.x, a.y); }
// a * b with explicit roundings (re = fma(a.x, b.x, -(a.y b.y)), im = fma(a.x, b.y, a.y b.x)),
// so the result does not depend on how the compiler contracts where this is inlined
__device__ __forceinline__ C2<float> cmul_rn(C2<float> a, C2<float> b) {
  return C2<float>{__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x))};
}
__device__ __forceinline__ C2<float> un(float2 a) { return C2<float>{a.x, a.y}; }
__device__ __forceinline__ C2<float> padd(C2<float> a, C2<float> b) { return un(__fadd2_rn(pk(a), pk(b))); }
// a - b as fma(b, -1, a): b * -1 is exact, so this is the correctly rounded difference
__device__ __forceinline__ C2<float> psub(C2<float> a, C2<float> b) {
  return un(__ffma2_rn(pk(b), make_float2(-1.f, -1.f), pk(a)));
}
__device__ __forceinline__ C2<float> pscale(float s, C2<float> a) { return un(__fmul2_rn(make_float2(s, s), pk(a))); }
// s * a + c
__device__ __forceinline__ C2<float> pfma(float s, C2<float> a, C2<float> c) {
  return un(__ffma2_rn(make_float2(s, s), pk(a), pk(c)));
}
// ---------------------------------------------------------------- rotations by three shears
// Multiplying by a twiddle exp(i theta) rounded to FP32 as (cos, sin) scales the value by
// |w| = 1 + O(2^-24), and for the few twiddles that a transform applies over and over
// (cos and sin of pi/8, sqrt(1/2)) the rounding leaves |w| below one: a 256-point
// transform then shrinks its output by about 2.6e-8 on average, and a forward and
// inverse 3D solve by about 1.5e-7, a systematic error of 1e-4 eV in the interaction
// energy of a 4 nm loop.  A rotation written as three shears,
//   x1 = x - t y,  y1 = y + s x1,  x2 = x1 - t y1,  t = tan(theta/2), s = sin(theta),
// has determinant one whatever the rounding of t and s, so its scale error vanishes to
// first order; each fma rounds once and without bias.  |theta| <= pi/2 keeps |t| <= 1;
// other angles are reduced by a half turn (g = -1, exact).  Same count as a complex
// multiply: three fma.  (Used for the compile-time twiddles of the register DFTs; the
// table twiddles are rounded so that their magnitude errors cancel, see the grid's
// table set-up.)
__device__ __forceinline__ C2<float> lift(C2<float> v, float t, float s) {
  const float x1 = __fmaf_rn(-t, v.y, v.x);
  const float y1 = __fmaf_rn(s, x1, v.y);
  const float x2 = __fmaf_rn(-t, y1, x1);
  return C2<float>{x2, y1};
}
// b + rot(e) and b - rot(e), rot = multiply by -i (forward) or +i (inverse)
template <bool INV> __device__ __forceinline__ C2<float> add_rot(C2<float> b, C2<float> e) {
  return INV ? C2<float>{b.x - e.y, b.y + e.x} : C2<float>{b.x + e.y, b.y - e.x};
}
template <bool INV> __device__ __forceinline__ C2<float> sub_rot(C2<float> b, C2<float> e) {
  return INV ? C2<float>{b.x + e.y, b.y - e.x} : C2<float>{b.x - e.y, b.y + e.x};
}
// b + s * rot(e) and b - s * rot(e)
template <bool INV> __device__ __forceinline__ C2<float> add_srot(C2<float> b, float s, C2<float> e) {
  return INV ? C2<float>{fmaf(-s, e.y, b.x), fmaf(s, e.x, b.y)} : C2<float>{fmaf(s, e.y, b.x), fmaf(-s, e.x, b.y)};
}
template <bool INV> __device__ __forceinline__ C2<float> sub_srot(C2<float> b, float s, C2<float> e) {
  return INV ? C2<float>{fmaf(s, e.y, b.x), fmaf(-s, e.x, b.y)} : C2<float>{fmaf(-s, e.y, b.x), fmaf(s, e.x, b.y)};
}

// ---------------------------------------------------------------- small DFTs
// X_k = sum_n x_n exp(-+2 pi i n k / R): minus sign forward, plus sign inverse.
template <class T, bool INV> __device__ __forceinline__ void dft2(C2<T>* v) {
  C2<T> a = v[0];
  v[0] = a + v[1];
  v[1] = a - v[1];
}
template <class T, bool INV> __device__ __forceinline__ void dft3(C2<T>* v) {
  const T s = T(0.86602540378443864676);  // sin(2 pi / 3)
  C2<T> t1 = v[1] + v[2], t2 = v[1] - v[2];
  C2<T> m = v[0] - T(0.5) * t1;
  C2<T> r = s * rot<T, INV>(t2);
  v[0] = v[0] + t1;
  v[1] = m + r;
  v[2] = m - r;
}
template <class T, bool INV> __device__ __forceinline__ void dft4(C2<T>* v) {
  C2<T> a = v[0] + v[2], b = v[0] - v[2], c = v[1] + v[3], d = rot<T, INV>(v[1] - v[3]);
  v[0] = a + c;
  v[2] = a - c;
  v[1] = b + d;
  v[3] = b - d;
}
template <class T, bool INV> __device__ __forceinline__ void dft5(C2<T>* v) {
  const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);  // cos(2pi/5), cos(4pi/5)
  const T s1 = T(0.95105651629515357212), s2 = T(0.58778525229247312917);   // sin(2pi/5), sin(4pi/5)
  C2<T> a1 = v[1] + v[4], b1 = v[1] - v[4], a2 = v[2] + v[3], b2 = v[2] - v[3];
  C2<T> m1 = v[0] + c1 * a1 + c2 * a2;
  C2<T> m2 = v[0] + c2 * a1 + c1 * a2;
  C2<T> n1 = rot<T, INV>(s1 * b1 + s2 * b2);
  C2<T> n2 = rot<T, INV>(s2 * b1 - s1 * b2);
  v[0] = v[0] + a1 + a2;
  v[1] = m1 + n1;
  v[4] = m1 - n1;
  v[2] = m2 + n2;
  v[3] = m2 - n2;
}
template <class T, bool INV> __device__ __forceinline__ void dft8(C2<T>* v) {
  const T h = T(0.70710678118654752440);  // sqrt(1/2)
  C2<T> e[4] = {v[0], v[2], v[4], v[6]};
  C2<T> o[4] = {v[1], v[3], v[5], v[7]};
  dft4<T, INV>(e);
  dft4<T, INV>(o);
  // twiddles w8^k, w8 = exp(-+ i pi/4)
  C2<T> o1 = INV ? C2<T>{h * (o[1].x - o[1].y), h * (o[1].x + o[1].y)}
                 : C2<T>{h * (o[1].x + o[1].y), h * (o[1].y - o[1].x)};
  C2<T> o2 = rot<T, INV>(o[2]);
  C2<T> o3 = INV ? C2<T>{h * (-o[3].x - o[3].y), h * (o[3].x - o[3].y)}
                 : C2<T>{h * (o[3].y - o[3].x), h * (-o[3].x - o[3].y)};
  v[0] = e[0] + o[0];
  v[4] = e[0] - o[0];
  v[1] = e[1] + o1;
  v[5] = e[1] - o1;
  v[2] = e[2] + o2;
  v[6] = e[2] - o2;
  v[3] = e[3] + o3;
  v[7] = e[3] - o3;
}
template <class T, bool INV, int R> __device__ __forceinline__ void dftR(C2<T>* v) {
  if constexpr (R == 2) dft2<T, INV>(v);
  else if constexpr (R == 3) dft3<T, INV>(v);
  else if constexpr (R == 4) dft4<T, INV>(v);
  else if constexpr (R == 5) dft5<T, INV>(v);
  else dft8<T, INV>(v);
}

// ---------------------------------------------------------------- line FFT engine
// A length-L transform runs as a sequence of Stockham autosort stages (the
// formulation of Govindaraju et al., SC'08) of radix 2, 3, 4, 5 or 8, one warp
// per line.  Stage s reads element j + r*(L/R), multiplies by w_L^(r*(j mod
// Ns)*L/(Ns*R)), does a radix-R DFT and writes element (j - j mod Ns)*R + j mod Ns
// + r*Ns, with Ns the product of the earlier radices; output is in natural order.
struct LinePlan {
  int L;
  int nst;
  int rad[8];
};

// Radix sequence of a length-L line (L = 2^a 3^b 5^c, L >= 4): radix 8 first, then a
// 4 or 4,4 for the leftover powers of two, then 3s and 5s; always two stages or more.
inline LinePlan make_plan(int L) {
  LinePlan p = {};
  p.L = L;
  int m = L, a = 0, b = 0, c = 0;
  while (m % 2 == 0) m /= 2, ++a;
  while (m % 3 == 0) m /= 3, ++b;
  while (m % 5 == 0) m /= 5, ++c;
  int r[16];
  int nr = 0;
  const int q = a / 3, rem = a % 3;
  if (rem == 0) {
    for (int i = 0; i < q; ++i) r[nr++] = 8;
  } else if (rem == 1) {
    if (q >= 1) {
      for (int i = 0; i < q - 1; ++i) r[nr++] = 8;
      r[nr++] = 4;
      r[nr++] = 4;
    } else {
      r[nr++] = 2;
    }
  } else {
    for (int i = 0; i < q; ++i) r[nr++] = 8;
    r[nr++] = 4;
  }
  for (int i = 0; i < b; ++i) r[nr++] = 3;
  for (int i = 0; i < c; ++i) r[nr++] = 5;
  if (nr == 1) {  // the engine wants two stages at least
    const int R = r[0];
    nr = 0;
    if (R == 8) { r[nr++] = 2; r[nr++] = 4; }
    else if (R == 4) { r[nr++] = 2; r[nr++] = 2; }
    else r[nr++] = R;
  }
  p.nst = nr;
  for (int i = 0; i < p.nst; ++i) p.rad[i] = r[i];
  return p;
}

template <class T>
struct SLine {  // strided line in shared, distributed-shared or global memory
  C2<T>* p;
  int s;
  __device__ __forceinline__ C2<T> ld(int i) const { return p[i * s]; }
  __device__ __forceinline__ void st(int i, C2<T> v) const { p[i * s] = v; }
};

template <class T, bool INV, int R, class In, class Out>
__device__ __forceinline__ void fft_stage(In in, Out out, const C2<T>* __restrict__ tw, int L, int Ns, int lane) {
  const int nb = L / R;
  const int tws = L / (Ns * R);
  for (int j = lane; j < nb; j += 32) {
    const int jm = j % Ns;
    C2<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in.ld(j + r * nb);
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C2<T> w = tw[r * jm * tws];
        if (INV) w.y = -w.y;
        v[r] = v[r] * w;
      }
    }
    dftR<T, INV, R>(v);
    const int o = (j - jm) * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) out.st(o + r * Ns, v[r]);
  }
}

template <class T, bool INV, class In, class Out>
__device__ __forceinline__ void fft_stage_any(int R, In in, Out out, const C2<T>* tw, int L, int Ns, int lane) {
  switch (R) {
    case 2: fft_stage<T, INV, 2>(in, out, tw, L, Ns, lane); break;
    case 3: fft_stage<T, INV, 3>(in, out, tw, L, Ns, lane); break;
    case 4: fft_stage<T, INV, 4>(in, out, tw, L, Ns, lane); break;
    case 5: fft_stage<T, INV, 5>(in, out, tw, L, Ns, lane); break;
    default: fft_stage<T, INV, 8>(in, out, tw, L, Ns, lane); break;
  }
}

// Transform of the line src into dst by one warp.  bufA/bufB: ping-pong lines of
// length L that alias neither src nor dst (bufB may alias src when src is a
// writable line that is no longer needed); plans have at least two stages.
template <class T, bool INV, class In, class Out>
__device__ void line_fft(In src, Out dst, C2<T>* bufA, C2<T>* bufB, const C2<T>* tw, const LinePlan& p, int lane) {
  SLine<T> a{bufA, 1}, b{bufB, 1};
  int Ns = 1;
  fft_stage_any<T, INV>(p.rad[0], src, a, tw, p.L, Ns, lane);
  __syncwarp();
  Ns *= p.rad[0];
  for (int s = 1; s < p.nst - 1; ++s) {
    if (s & 1) fft_stage_any<T, INV>(p.rad[s], a, b, tw, p.L, Ns, lane);
    else fft_stage_any<T, INV>(p.rad[s], b, a, tw, p.L, Ns, lane);
    __syncwarp();
    Ns *= p.rad[s];
  }
  if ((p.nst - 2) & 1) fft_stage_any<T, INV>(p.rad[p.nst - 1], b, dst, tw, p.L, Ns, lane);
  else fft_stage_any<T, INV>(p.rad[p.nst - 1], a, dst, tw, p.L, Ns, lane);
  __syncwarp();
}

// ---------------------------------------------------------------- pass configuration
struct PassCfg {
  int nx, ny, nz, H;   // H = nx/2
  int ncomp;           // components (planes per z)
  int cs;              // cluster size of the plane passes
  int tw_w;            // pencil tile width (consecutive ky per kx)
  int k0_mode;
  int forward_only;    // pencil pass: stop after the forward z transform
  double q;            // fixed-point quantum of the eigenstrain input
  double C11, C12, C44;
  float fC[3];         // C11, C12, C44 rounded to FP32 (the FP32 Green operator's constants)
  float fCs[3];        // C11, C12, C44 / (nx ny nz), rounded to FP32 once from FP64
  LinePlan pH, pY, pZ;
  const void* twH;     // C2<T>[H]      w_H^k
  const void* twY;     // C2<T>[ny]
  const void* twZ;     // C2<T>[nz]
  const void* untw;    // C2<T>[H+1]    exp(-2 pi i k / nx)
  // the same twiddles for the FP32 register-FFT passes, each rounded to the FP32 pair
  // whose magnitude error keeps the running sum of the table's errors near zero:
  const void* ftwH;    // C2<float>[H]   w_H^m
  const void* ftwY;    // C2<float>[ny]
  const void* ftwZ;    // C2<float>[nz]
  const void* ftwU;    // C2<float>[H+1] exp(-2 pi i k / nx)
  int* err;            // device error word (bounded waits that gave up set it)
  float rn[3];         // 1/nx, 1/ny, 1/nz (rounded from FP64)
  int* dirty;          // fast forward plane pass: per plane (c*nz + z) flag, nonzero when the
                       // plane's eigenstrain changed since its last transform (the pass skips
                       // clean planes and clears the flags it consumed); nullptr: every plane
  int tx_extra;        // bytes a TMA-staged pass expects beyond its copies: 0, except where a
                       // test makes that pass's bounded wait run out
};

// ---------------------------------------------------------------- defects
struct DefGeo {
  double e6[6];       // eigenstrain tensor (xx, yy, zz, yz, xz, xy)
  double escale;      // e6 = escale * (pattern of 0 and +-1): |b|/(h |a|^2) for loops, the dilatation
  float ew[6];        // energy weights e6 / escale with the off-diagonals doubled (0, +-1, +-2: exact)
  double v_over_h3;   // shape volume / h^3
  double thr;         // disk: |a|^2 (8R/h)^2; sphere: (8 rho)^6
  int kind;           // 0 disk, 1 sphere
  int a[3];           // disk axis (integer vector)
  int a2;
  int extent;         // scan half-width in voxels
  int allowed;        // bit j set: jump j allowed
  int z;              // number of allowed jumps
};

struct Move {
  int i;
  int old_pos[3];
  int new_pos[3];
};

// Kinetic state kept on the device (one per handle).
struct DevState {
  double clock;
  double dt_last;
  long long events;
  long long negative_barriers;
  long long step;
  int nmoves;
  int err;
  double dt_fixed;
};

// Optional rate output of the energies kernel (rates == nullptr: energies only).
struct RateArgs {
  double* rates;        // [n][8] biased jump frequencies (0 for jumps not allowed)
  double* rsum;         // [n] sum over j
  long long* negb;      // count of negative effective barriers
  double nu0, kT;
  double rkT;           // 1 / kT
};

// Eigenstrain tensors of the (at most three) defects whose self terms one batch computes.
// One batch of the self-term build: up to three defects (the stencils of defect
// idx[d] in classes 0 and 1 occupy fields 2d and 2d+1), the type table row of each
// and the square of its eigenstrain scale relative to the type's unit tensor.
struct WBatch {
  int idx[3];
  int type[3];
  double s2[3];
  int nb;
};

// Energy lists (one per defect and current class; ptr < 0: none, the energies kernel
// then walks the site stencil once and the candidate stencil eight times): every voxel
// of the site stencil or of a candidate stencil, once, with its nine counts.
struct DilatedLists {
  const int* ptr;                 // [2 nd] first entry of list (i, c)
  const int* end;                 // [2 nd] one past the last entry
  const int* off;                 // packed offsets of the voxels (relative to the site's base voxel)
  const unsigned long long* cnt;  // counts of the eight candidates, byte j for jump j
  const uint8_t* scnt;            // count of the site stencil
};

// Energies by fixed chunks of the energy lists: defect i owns the chunk slots
// c0[i] .. c0[i] + ceil(max(len(i, 0), len(i, 1)) / kEnergyWarpEntries) - 1, of which its
// current site class c uses the first ceil(len(i, c) / kEnergyWarpEntries); slot w holds
// entries c0 + w * kEnergyWarpEntries on of the class-c list.  One warp sums one chunk
// into part[w][9] (site, then the eight jumps), and the finishing pass adds a defect's
// chunks in slot order.
struct ChunkArgs {
  const int* cdef;  // [nchunk] the defect of each slot
  const int* c0;    // [nd] the first slot of each defect
  double* part;     // [nchunk][9] chunk sums
  int nchunk;
};

// Unit eigenstrain tensors of the defect types present (at most eight: four
// 1/2<111> loop axes, three <100> loop axes, the dilatational SIA cluster).
struct QTypes {
  double e6[8][6];
  int nt;
};

// The energies kernel: a block of kEnergyThreads threads per defect whose energy list is
// longer than kEnergyWarpEntries entries, one warp per defect otherwise.
constexpr int kEnergyThreads = 256;
constexpr int kEnergyWarpEntries = 128;

// One replica of a batched ensemble as the batched kernels see it (an array of these
// lives in device memory): the pass configuration and buffers of its FP32 register-FFT
// solve, and the defect-side arrays of its step.  Work lists pair a replica index with
// a plane, a pencil tile or a defect (in the energies kernel's order).
struct BatchRep {
  PassCfg cfg;                // dirty flags set (the forward pass skips clean planes)
  const int32_t* eps;         // fixed-point eigenstrain
  C2<float>* spec;            // plane transforms of the eigenstrain (kept between solves)
  C2<float>* spec2;           // Green operator output
  float* sig;                 // stress
  okmc_defect* def;
  const DefGeo* geo;
  const int* ptr;
  const int* off;
  const uint8_t* cnt;
  const double* alpha;
  const double* W;
  const int* order;           // energies: defects largest stencil first
  double* E;
  double* Ec;
  RateArgs ra;
  DilatedLists dl;
  ChunkArgs ca;               // energies by chunks of the energy lists
  double pref;                // -kappa h^3
  double nu0, kT;
  Move* moves;
  DevState* state;
  int* err;
  double rq, lim;             // fixed-point scale and limit of the eigenstrain
  uint32_t key0, key1;        // Philox key (the grid's seed)
  int3 n;
  int nd;
  int mode;                   // OKMC_RESIDENCE or OKMC_FIXED_DT
};

__host__ __device__ __forceinline__ int pack_off(int dx, int dy, int dz) {
  return (dx + 512) | ((dy + 512) << 10) | ((dz + 512) << 20);
}
__host__ __device__ __forceinline__ void unpack_off(int p, int& dx, int& dy, int& dz) {
  dx = (p & 1023) - 512;
  dy = ((p >> 10) & 1023) - 512;
  dz = ((p >> 20) & 1023) - 512;
}

__host__ __device__ __forceinline__ int floor_div2(int p) { return p >= 0 ? p / 2 : -((1 - p) / 2); }

// jump j <-> (sx, sy, sz), j = 4(sx>0) + 2(sy>0) + (sz>0)
__host__ __device__ __forceinline__ int jump_comp(int j, int a) { return ((j >> (2 - a)) & 1) ? 1 : -1; }

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
__host__ __device__ __forceinline__ void philox4x32_10(const uint32_t ctr_in[4], uint32_t k0, uint32_t k1, uint32_t out[4]) {
  uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * x0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    x0 = hi1 ^ x1 ^ k0;
    x1 = lo1;
    x2 = hi0 ^ x3 ^ k1;
    x3 = lo0;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}
// uniform on (0, 1]: ((hi << 21) | (lo >> 11)) + 1 over 2^53
__host__ __device__ __forceinline__ double u53(uint32_t lo, uint32_t hi) {
  const uint64_t k = (((uint64_t)hi << 21) | (lo >> 11)) + 1ull;
  return (double)k * 1.1102230246251565404e-16;
}

// ---------------------------------------------------------------- Green operator
template <class T>
struct GreenC {
  T C11, C12, C44;
};

// sigma_hat = C:(sym(q (x) K(q)^-1 (tau q)) - eps*_hat), tau = C:eps*_hat, K_ik = C_ijkl q_j q_l,
// for cubic C (paper Eqs. EIG_elastic_fourier, basicgammacomplete, summaryEL with the
// standard index reading of Gamma).  Gamma is homogeneous of degree 0 in the
// frequency, so q need not be normalised.  The polarisation uses Cs = C/N so that
// the result comes out already scaled by 1/N; K and the final C:(...) use C.
template <class T>
__device__ __forceinline__ void sigma_of(const C2<T>* e, T q0, T q1, T q2, const GreenC<T>& C, const GreenC<T>& Cs,
                                         C2<T>* s) {
  const T ds = Cs.C11 - Cs.C12, gs = T(2) * Cs.C44;
  const C2<T> tr = e[0] + e[1] + e[2];
  const C2<T> t0 = Cs.C12 * tr + ds * e[0], t1 = Cs.C12 * tr + ds * e[1], t2 = Cs.C12 * tr + ds * e[2];
  const C2<T> t3 = gs * e[3], t4 = gs * e[4], t5 = gs * e[5];
  const C2<T> v0 = q0 * t0 + q1 * t5 + q2 * t4;
  const C2<T> v1 = q0 * t5 + q1 * t1 + q2 * t3;
  const C2<T> v2 = q0 * t4 + q1 * t3 + q2 * t2;
  const T A = C.C11 - C.C12 - T(2) * C.C44, B = C.C12 + C.C44;
  const T a0 = q0 * q0, a1 = q1 * q1, a2 = q2 * q2;
  const T cq = C.C44 * (a0 + a1 + a2);
  const T k00 = cq + (A + B) * a0, k11 = cq + (A + B) * a1, k22 = cq + (A + B) * a2;
  const T k01 = B * q0 * q1, k02 = B * q0 * q2, k12 = B * q1 * q2;
  const T i00 = k11 * k22 - k12 * k12, i01 = k02 * k12 - k01 * k22, i02 = k01 * k12 - k02 * k11;
  const T i11 = k00 * k22 - k02 * k02, i12 = k01 * k02 - k00 * k12, i22 = k00 * k11 - k01 * k01;
  const T rdet = T(1) / (k00 * i00 + k01 * i01 + k02 * i02);
  const C2<T> w0 = rdet * (i00 * v0 + i01 * v1 + i02 * v2);
  const C2<T> w1 = rdet * (i01 * v0 + i11 * v1 + i12 * v2);
  const C2<T> w2 = rdet * (i02 * v0 + i12 * v1 + i22 * v2);
  const C2<T> qw = q0 * w0 + q1 * w1 + q2 * w2;
  const T d = C.C11 - C.C12;
  s[0] = C.C12 * qw + d * (q0 * w0) - t0;
  s[1] = C.C12 * qw + d * (q1 * w1) - t1;
  s[2] = C.C12 * qw + d * (q2 * w2) - t2;
  s[3] = C.C44 * (q1 * w2 + q2 * w1) - t3;
  s[4] = C.C44 * (q0 * w2 + q2 * w0) - t4;
  s[5] = C.C44 * (q0 * w1 + q1 * w0) - t5;
}

// The same for FP32 on paired instructions: every complex-times-real term is one
// packed fma; the adjugate and the determinant stay scalar.  Every operation is an
// explicit intrinsic, so the rounding does not depend on how the compiler contracts
// products and sums where this is inlined (launch variants agree bit for bit).
//
// The operator annihilates compatible strains, sym(q (x) a) for any vector a, so it is
// applied to the transverse part eta = e - sym(q (x) a) with a chosen such that
// eta q = 0: a = (2 e q - (q.e.q / |q|^2) q) / |q|^2.  For the one-voxel-thick loops
// nearly all of e is compatible at the frequencies that carry their spectrum, and
// C:sym(q (x) w) and tau = C:e then cancel to a few percent.  Applied to e itself, the
// rounding of those two large terms is an error on the output side, at the scale of
// the loop's unrelaxed energy (about 30 times its elastic energy for a 4 nm loop).
// Applied to eta, every intermediate is of the size of the result; the rounding of
// eta itself acts as a perturbation of the input, which the operator then maps
// exactly, and which pairs with the (small) relaxed field of any defect.
// 1/x by the hardware approximation (about one ulp; deterministic, so launch variants
// still agree bit for bit).  Used where a relative error of one ulp in the reciprocal only
// rescales a term that is of the size of the result: 1/|q|^2 of the transverse split (an
// input-side perturbation the operator maps exactly) and 1/det K (the compatible
// correction w, of the size of the elastic field once e is transverse).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void sigma_of(const C2<float>* e_in, float q0, float q1, float q2, const GreenC<float>& C,
                                         const GreenC<float>& Cs, C2<float>* s) {
  C2<float> e[6];
  {
    const float qq = __fmaf_rn(q2, q2, __fmaf_rn(q1, q1, __fmul_rn(q0, q0)));
    const float rqq = rcp_approx(qq);
    const C2<float> u0 = pfma(q2, e_in[4], pfma(q1, e_in[5], pscale(q0, e_in[0])));
    const C2<float> u1 = pfma(q2, e_in[3], pfma(q1, e_in[1], pscale(q0, e_in[5])));
    const C2<float> u2 = pfma(q2, e_in[2], pfma(q1, e_in[3], pscale(q0, e_in[4])));
    // r = (q.e.q) / |q|^2; a_i = (2 u_i - r q_i) / |q|^2
    const C2<float> r = pscale(rqq, pfma(q2, u2, pfma(q1, u1, pscale(q0, u0))));
    const C2<float> a0 = pscale(rqq, pfma(-q0, r, pscale(2.f, u0)));
    const C2<float> a1 = pscale(rqq, pfma(-q1, r, pscale(2.f, u1)));
    const C2<float> a2 = pscale(rqq, pfma(-q2, r, pscale(2.f, u2)));
    e[0] = pfma(-q0, a0, e_in[0]);
    e[1] = pfma(-q1, a1, e_in[1]);
    e[2] = pfma(-q2, a2, e_in[2]);
    e[3] = pfma(-0.5f, pfma(q1, a2, pscale(q2, a1)), e_in[3]);
    e[4] = pfma(-0.5f, pfma(q0, a2, pscale(q2, a0)), e_in[4]);
    e[5] = pfma(-0.5f, pfma(q0, a1, pscale(q1, a0)), e_in[5]);
  }
  const float ds = __fsub_rn(Cs.C11, Cs.C12), gs = __fmul_rn(2.f, Cs.C44);
  const C2<float> tr = padd(padd(e[0], e[1]), e[2]);
  const C2<float> c12tr = pscale(Cs.C12, tr);
  const C2<float> t0 = pfma(ds, e[0], c12tr), t1 = pfma(ds, e[1], c12tr), t2 = pfma(ds, e[2], c12tr);
  const C2<float> t3 = pscale(gs, e[3]), t4 = pscale(gs, e[4]), t5 = pscale(gs, e[5]);
  const C2<float> v0 = pfma(q2, t4, pfma(q1, t5, pscale(q0, t0)));
  const C2<float> v1 = pfma(q2, t3, pfma(q1, t1, pscale(q0, t5)));
  const C2<float> v2 = pfma(q2, t2, pfma(q1, t3, pscale(q0, t4)));
  const float B = __fadd_rn(C.C12, C.C44);
  const float AB = __fsub_rn(C.C11, C.C44);  // A + B with A = C11 - C12 - 2 C44
  const float a0 = __fmul_rn(q0, q0), a1 = __fmul_rn(q1, q1), a2 = __fmul_rn(q2, q2);
  const float cq = __fmul_rn(C.C44, __fadd_rn(__fadd_rn(a0, a1), a2));
  const float k00 = __fmaf_rn(AB, a0, cq), k11 = __fmaf_rn(AB, a1, cq), k22 = __fmaf_rn(AB, a2, cq);
  const float Bq0 = __fmul_rn(B, q0);
  const float k01 = __fmul_rn(Bq0, q1), k02 = __fmul_rn(Bq0, q2), k12 = __fmul_rn(__fmul_rn(B, q1), q2);
  // a*b - c*d as fma(a, b, -(c*d))
  auto dif = [](float a, float b, float c, float d) { return __fmaf_rn(a, b, -__fmul_rn(c, d)); };
  const float i00 = dif(k11, k22, k12, k12), i01 = dif(k02, k12, k01, k22), i02 = dif(k01, k12, k02, k11);
  const float i11 = dif(k00, k22, k02, k02), i12 = dif(k01, k02, k00, k12), i22 = dif(k00, k11, k01, k01);
  const float rdet = rcp_approx(__fmaf_rn(k02, i02, __fmaf_rn(k01, i01, __fmul_rn(k00, i00))));
  const C2<float> w0 = pscale(rdet, pfma(i02, v2, pfma(i01, v1, pscale(i00, v0))));
  const C2<float> w1 = pscale(rdet, pfma(i12, v2, pfma(i11, v1, pscale(i01, v0))));
  const C2<float> w2 = pscale(rdet, pfma(i22, v2, pfma(i12, v1, pscale(i02, v0))));
  const C2<float> qw = pfma(q2, w2, pfma(q1, w1, pscale(q0, w0)));
  const float d = __fsub_rn(C.C11, C.C12);
  const C2<float> c12qw = pscale(C.C12, qw);
  s[0] = pfma(__fmul_rn(d, q0), w0, psub(c12qw, t0));
  s[1] = pfma(__fmul_rn(d, q1), w1, psub(c12qw, t1));
  s[2] = pfma(__fmul_rn(d, q2), w2, psub(c12qw, t2));
  s[3] = psub(pscale(C.C44, pfma(q1, w2, pscale(q2, w1))), t3);
  s[4] = psub(pscale(C.C44, pfma(q0, w2, pscale(q2, w0))), t4);
  s[5] = psub(pscale(C.C44, pfma(q0, w1, pscale(q1, w0))), t5);
}

// Green operator at half-spectrum index (kx, ky, kz), in place on e[6], scaled by
// 1/N.  Frequencies follow Eq. frequencies (n = k for k < N/2, k - N otherwise,
// so the Nyquist index is -N/2); on Nyquist planes the operator is averaged over
// the sign of the Nyquist components, which is what the real part of the inverse
// of the full spectrum computes.
// scale: 1/N (the solve) or 1 (unnormalised spectra).  The FP32 constants come ready from
// the pass configuration, so no FP64 arithmetic or conversion runs per frequency (the FP64
// pipe of this GPU is narrow, and the compiler may re-derive hoisted values per call).
template <class T>
__device__ __forceinline__ void green_point(C2<T>* e, int kx, int ky, int kz, const PassCfg& c, T scale) {
  GreenC<T> C, Cs;
  if constexpr (sizeof(T) == 4) {
    C = GreenC<T>{c.fC[0], c.fC[1], c.fC[2]};
    Cs = scale == T(1) ? C : GreenC<T>{c.fCs[0], c.fCs[1], c.fCs[2]};
  } else {
    C = GreenC<T>{T(c.C11), T(c.C12), T(c.C44)};
    Cs = GreenC<T>{T(c.C11 * (double)scale), T(c.C12 * (double)scale), T(c.C44 * (double)scale)};
  }
  const int fx = kx < c.H ? kx : kx - c.nx;
  const int fy = ky < c.ny / 2 ? ky : ky - c.ny;
  const int fz = kz < c.nz / 2 ? kz : kz - c.nz;
  if (fx == 0 && fy == 0 && fz == 0) {
    if (c.k0_mode == OKMC_MEAN_STRAIN_ZERO) {
      if constexpr (sizeof(T) == 4) {  // explicit roundings, as in sigma_of
        const float ds = __fsub_rn(Cs.C11, Cs.C12), gs = __fmul_rn(2.f, Cs.C44);
        const C2<float> c12tr = pscale(Cs.C12, padd(padd(e[0], e[1]), e[2]));
        const C2<float> t0 = pfma(ds, e[0], c12tr), t1 = pfma(ds, e[1], c12tr), t2 = pfma(ds, e[2], c12tr);
        e[0] = pscale(-1.f, t0);
        e[1] = pscale(-1.f, t1);
        e[2] = pscale(-1.f, t2);
        for (int a = 3; a < 6; ++a) e[a] = pscale(-gs, e[a]);
      } else {
        const T ds = Cs.C11 - Cs.C12, gs = T(2) * Cs.C44;
        const C2<T> tr = e[0] + e[1] + e[2];
        const C2<T> t0 = Cs.C12 * tr + ds * e[0], t1 = Cs.C12 * tr + ds * e[1], t2 = Cs.C12 * tr + ds * e[2];
        e[0] = T(-1) * t0;
        e[1] = T(-1) * t1;
        e[2] = T(-1) * t2;
        for (int a = 3; a < 6; ++a) e[a] = (-gs) * e[a];
      }
    } else {
      for (int a = 0; a < 6; ++a) e[a] = C2<T>{T(0), T(0)};
    }
    return;
  }
  // FP32: multiply by the reciprocal edge; FP64: divide (the reciprocals are FP32)
  T q0, q1, q2;
  if constexpr (sizeof(T) == 4) {
    q0 = T(fx) * c.rn[0];
    q1 = T(fy) * c.rn[1];
    q2 = T(fz) * c.rn[2];
  } else {
    q0 = T(fx) / T(c.nx);
    q1 = T(fy) / T(c.ny);
    q2 = T(fz) / T(c.nz);
  }
  C2<T> s[6];
  sigma_of(e, q0, q1, q2, C, Cs, s);
  const bool nx_ = (kx == c.H), ny_ = (2 * ky == c.ny), nz_ = (2 * kz == c.nz);
  if (nx_ || ny_ || nz_) {
    C2<T> s2[6];
    sigma_of(e, nx_ ? -q0 : q0, ny_ ? -q1 : q1, nz_ ? -q2 : q2, C, Cs, s2);
    for (int a = 0; a < 6; ++a) s[a] = T(0.5) * (s[a] + s2[a]);
  }
  for (int a = 0; a < 6; ++a) e[a] = s[a];
}

}  // namespace okmc
