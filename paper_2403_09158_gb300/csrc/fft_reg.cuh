// Register-resident line FFTs for power-of-two lengths 16..256 (FP32).
//
// A line of length L = R1*R2 is transformed by a group of NT = min(R1, R2)
// consecutive threads of one warp in two steps (Cooley-Tukey, n = n1 + R1*n2,
// k = k2 + R2*k1):
//   step 1: for each n1, a length-R2 DFT over n2 of x[n1 + R1*n2] in registers,
//           times the twiddle w_L^(n1*k2), written to an exchange slot (n1, k2);
//   step 2: for each k2, a length-R1 DFT over n1 of the slots (n1, k2), giving
//           X[k2 + R2*k1] in natural order.
// Every thread loads all of its inputs before any write, so the input line, the
// exchange slots and the output may share memory; the warp synchronises between
// the phases (all 32 lanes must call, inactive groups pass active = false).
#pragma once

#include "okmc_internal.cuh"

namespace okmc {

template <int L> struct RegPlan;
template <> struct RegPlan<16> { static constexpr int R1 = 4, R2 = 4; };
template <> struct RegPlan<32> { static constexpr int R1 = 4, R2 = 8; };
template <> struct RegPlan<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct RegPlan<128> { static constexpr int R1 = 8, R2 = 16; };
template <> struct RegPlan<256> { static constexpr int R1 = 16, R2 = 16; };
template <int L> __host__ __device__ constexpr int reg_nt() { return RegPlan<L>::R1 < RegPlan<L>::R2 ? RegPlan<L>::R1 : RegPlan<L>::R2; }

// cos and sin of 2 pi e / 16 for e = 0..15
__device__ __forceinline__ float cos16(int e) {
  switch (e & 15) {
    case 0: return 1.0f;
    case 1: return 0.92387953251128676f;
    case 2: return 0.70710678118654752f;
    case 3: return 0.38268343236508977f;
    case 4: return 0.0f;
    case 5: return -0.38268343236508977f;
    case 6: return -0.70710678118654752f;
    case 7: return -0.92387953251128676f;
    case 8: return -1.0f;
    case 9: return -0.92387953251128676f;
    case 10: return -0.70710678118654752f;
    case 11: return -0.38268343236508977f;
    case 12: return 0.0f;
    case 13: return 0.38268343236508977f;
    case 14: return 0.70710678118654752f;
    default: return 0.92387953251128676f;
  }
}
__device__ __forceinline__ float sin16(int e) { return cos16(e - 4); }

// v * exp(-+2 pi i e / 16) with the trivial exponents kept exact
template <bool INV>
__device__ __forceinline__ C2<float> tw16(C2<float> v, int e) {
  e &= 15;
  if (e == 0) return v;
  if (e == 4) return rot<float, INV>(v);
  if (e == 8) return C2<float>{-v.x, -v.y};
  if (e == 12) return rot<float, !INV>(v);
  const float c = cos16(e), s = INV ? sin16(e) : -sin16(e);
  return C2<float>{v.x * c - v.y * s, v.x * s + v.y * c};
}

template <bool INV>
__device__ __forceinline__ void dft16(C2<float>* v) {
  C2<float> y[16];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    C2<float> a[4] = {v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]};
    dft4<float, INV>(a);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) y[n1 * 4 + k2] = tw16<INV>(a[k2], n1 * k2);
  }
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    C2<float> b[4] = {y[k2], y[4 + k2], y[8 + k2], y[12 + k2]};
    dft4<float, INV>(b);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) v[k2 + 4 * k1] = b[k1];
  }
}

template <int R, bool INV>
__device__ __forceinline__ void dft_reg(C2<float>* v) {
  if constexpr (R == 4) dft4<float, INV>(v);
  else if constexpr (R == 8) dft8<float, INV>(v);
  else dft16<INV>(v);
}

// exchange slots: padded [R1][R2 + 1] rows
template <int R2>
struct XPad {
  C2<float>* p;
  __device__ __forceinline__ C2<float>& operator()(int n1, int k2) const { return p[n1 * (R2 + 1) + k2]; }
};
// exchange slots inside a strided line of L elements, skewed so that both the row
// writes and the column reads hit distinct banks
template <int R2>
struct XSkew {
  C2<float>* p;
  int s;
  __device__ __forceinline__ C2<float>& operator()(int n1, int k2) const {
    return p[s * (n1 * R2 + ((k2 + n1) & (R2 - 1)))];
  }
};

// Twiddles w_L^(n1*k2) as a padded [R1][R2 + 1] table: a warp's threads (consecutive
// n1, one k2) then read distinct banks.  tw2 is filled by fill_tw2 from w_L^k.
template <int L>
__host__ __device__ constexpr int tw2_size() { return RegPlan<L>::R1 * (RegPlan<L>::R2 + 1); }
template <int L>
__device__ __forceinline__ void fill_tw2(C2<float>* tw2, const C2<float>* __restrict__ tw) {
  constexpr int R2 = RegPlan<L>::R2;
  for (int i = threadIdx.x; i < tw2_size<L>(); i += blockDim.x) {
    const int n1 = i / (R2 + 1), k2 = i % (R2 + 1);
    tw2[i] = k2 < R2 ? tw[n1 * k2] : C2<float>{1.f, 0.f};
  }
}

template <bool INV, int L, class Ld, class Xch, class St>
__device__ __forceinline__ void reg_fft(const Ld& ld, const Xch& x, const St& st, const C2<float>* __restrict__ tw2, int t,
                                        bool active) {
  constexpr int R1 = RegPlan<L>::R1, R2 = RegPlan<L>::R2, NT = reg_nt<L>();
  constexpr int A = R1 / NT, B = R2 / NT;
  C2<float> v[A][R2];
  if (active) {
#pragma unroll
    for (int a = 0; a < A; ++a)
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) v[a][n2] = ld(t + NT * a + R1 * n2);
  }
  __syncwarp();
  if (active) {
#pragma unroll
    for (int a = 0; a < A; ++a) {
      const int n1 = t + NT * a;
      dft_reg<R2, INV>(v[a]);
      x(n1, 0) = v[a][0];
#pragma unroll
      for (int k2 = 1; k2 < R2; ++k2) {
        C2<float> w = tw2[n1 * (R2 + 1) + k2];
        if (INV) w.y = -w.y;
        x(n1, k2) = v[a][k2] * w;
      }
    }
  }
  __syncwarp();
  C2<float> u[B][R1];
  if (active) {
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) u[b][n1] = x(n1, t + NT * b);
  }
  __syncwarp();
  if (active) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      dft_reg<R1, INV>(u[b]);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) st(t + NT * b + R2 * k1, u[b][k1]);
    }
  }
  __syncwarp();
}

}  // namespace okmc
