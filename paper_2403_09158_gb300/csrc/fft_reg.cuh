// Register-resident line FFTs (FP32) for lengths 16..320 of the form 2^a 3^b 5^c used by
// the fast passes.
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

// L = R1 * R2 with R1 <= R2; NT = R1 threads per line; each thread does one length-R2
// DFT in step 1 and ceil(R2 / R1) length-R1 DFTs in step 2 (the last round partial
// when R1 does not divide R2).
template <int L> struct RegPlan;
template <> struct RegPlan<16> { static constexpr int R1 = 4, R2 = 4; };
template <> struct RegPlan<24> { static constexpr int R1 = 4, R2 = 6; };
template <> struct RegPlan<32> { static constexpr int R1 = 4, R2 = 8; };
template <> struct RegPlan<48> { static constexpr int R1 = 4, R2 = 12; };
template <> struct RegPlan<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct RegPlan<80> { static constexpr int R1 = 4, R2 = 20; };
template <> struct RegPlan<96> { static constexpr int R1 = 8, R2 = 12; };
template <> struct RegPlan<128> { static constexpr int R1 = 8, R2 = 16; };
template <> struct RegPlan<160> { static constexpr int R1 = 8, R2 = 20; };
template <> struct RegPlan<192> { static constexpr int R1 = 8, R2 = 24; };
template <> struct RegPlan<256> { static constexpr int R1 = 16, R2 = 16; };
template <> struct RegPlan<320> { static constexpr int R1 = 16, R2 = 20; };
template <int L> __host__ __device__ constexpr int reg_nt() { return RegPlan<L>::R1 < RegPlan<L>::R2 ? RegPlan<L>::R1 : RegPlan<L>::R2; }
// (R1, R2) of a register-FFT length known only at run time (host code); false if L has no plan
inline bool reg_split(int L, int& R1, int& R2) {
  switch (L) {
#define OKMC_SPLIT(n) \
  case n: R1 = RegPlan<n>::R1; R2 = RegPlan<n>::R2; return true;
    OKMC_SPLIT(16) OKMC_SPLIT(24) OKMC_SPLIT(32) OKMC_SPLIT(48) OKMC_SPLIT(64) OKMC_SPLIT(80) OKMC_SPLIT(96)
    OKMC_SPLIT(128) OKMC_SPLIT(160) OKMC_SPLIT(192) OKMC_SPLIT(256) OKMC_SPLIT(320)
#undef OKMC_SPLIT
    default: return false;
  }
}

// Small DFTs on packed pairs; X_k = sum_n x_n exp(-+2 pi i n k / R), minus sign forward.
template <bool INV> __device__ __forceinline__ void pdft2(C2<float>* v) {
  const C2<float> a = v[0];
  v[0] = padd(a, v[1]);
  v[1] = psub(a, v[1]);
}
template <bool INV> __device__ __forceinline__ void pdft3(C2<float>* v) {
  const float s = 0.86602540378443864676f;  // sin(2 pi / 3)
  const C2<float> t1 = padd(v[1], v[2]), t2 = psub(v[1], v[2]);
  const C2<float> m = pfma(-0.5f, t1, v[0]);
  v[0] = padd(v[0], t1);
  v[1] = add_srot<INV>(m, s, t2);
  v[2] = sub_srot<INV>(m, s, t2);
}
template <bool INV> __device__ __forceinline__ void pdft4(C2<float>* v) {
  const C2<float> a = padd(v[0], v[2]), b = psub(v[0], v[2]), c = padd(v[1], v[3]), e = psub(v[1], v[3]);
  v[0] = padd(a, c);
  v[2] = psub(a, c);
  v[1] = add_rot<INV>(b, e);
  v[3] = sub_rot<INV>(b, e);
}
template <bool INV> __device__ __forceinline__ void pdft5(C2<float>* v) {
  const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;  // cos(2pi/5), cos(4pi/5)
  const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;   // sin(2pi/5), sin(4pi/5)
  const C2<float> a1 = padd(v[1], v[4]), b1 = psub(v[1], v[4]), a2 = padd(v[2], v[3]), b2 = psub(v[2], v[3]);
  const C2<float> m1 = pfma(c2, a2, pfma(c1, a1, v[0]));
  const C2<float> m2 = pfma(c1, a2, pfma(c2, a1, v[0]));
  const C2<float> n1 = pfma(s2, b2, pscale(s1, b1));
  const C2<float> n2 = pfma(-s1, b2, pscale(s2, b1));
  v[0] = padd(v[0], padd(a1, a2));
  v[1] = add_rot<INV>(m1, n1);
  v[4] = sub_rot<INV>(m1, n1);
  v[2] = add_rot<INV>(m2, n2);
  v[3] = sub_rot<INV>(m2, n2);
}
// tan(pi j / 240) and sin(2 pi j / 240) for the j that the compile-time twiddles use
// (multiples of 240/R for R = 6, 8, 10, 12, 16, 20, 24, up to a quarter turn)
__device__ __forceinline__ float tan240(int j) {
  switch (j) {
    case 10: return 0.1316524975873958534715f;
    case 12: return 0.1583844403245362938388f;
    case 15: return 0.1989123673796580069115f;
    case 20: return 0.2679491924311227064725f;
    case 24: return 0.3249196962329063261558f;
    case 30: return 0.4142135623730950488016f;
    case 36: return 0.5095254494944288105137f;
    case 40: return 0.5773502691896257645091f;
    case 45: return 0.6681786379192989199977f;
    case 48: return 0.7265425280053608858954f;
    case 50: return 0.7673269879789603429230f;
    case 60: return 1.0000000000000000000000f;
    default: return 0.0f;
  }
}
__device__ __forceinline__ float sin240(int j) {
  switch (j) {
    case 10: return 0.2588190451025207623488f;
    case 12: return 0.3090169943749474241022f;
    case 15: return 0.3826834323650897717284f;
    case 20: return 0.5000000000000000000000f;
    case 24: return 0.5877852522924731291687f;
    case 30: return 0.7071067811865475244008f;
    case 36: return 0.8090169943749474241022f;
    case 40: return 0.8660254037844386467637f;
    case 45: return 0.9238795325112867561281f;
    case 48: return 0.9510565162951535721164f;
    case 50: return 0.9659258262890682867497f;
    case 60: return 1.0000000000000000000000f;
    default: return 0.0f;
  }
}

// v * exp(-+2 pi i e / R) (minus sign forward) for a compile-time e and R dividing 240:
// quarter turns exactly, any other angle as a rotation by three shears (lift).
template <int R, bool INV>
__device__ __forceinline__ C2<float> twc(C2<float> v, int e) {
  e %= R;
  if (e == 0) return v;
  if (4 * e == R) return rot<float, INV>(v);
  if (2 * e == R) return C2<float>{-v.x, -v.y};
  if (4 * e == 3 * R) return rot<float, !INV>(v);
  int j = -e * (240 / R);  // forward angle in units of 2 pi / 240, in (-240, 0)
  if (j <= -120) j += 240;  // (-120, 120]
  bool neg = false;
  if (j < -60) {
    j += 120;
    neg = true;
  } else if (j > 60) {
    j -= 120;
    neg = true;
  }
  if (INV) j = -j;
  const float t = j >= 0 ? tan240(j) : -tan240(-j);
  const float s = j >= 0 ? sin240(j) : -sin240(-j);
  const C2<float> r = lift(v, t, s);
  return neg ? C2<float>{-r.x, -r.y} : r;
}

template <bool INV> __device__ __forceinline__ void pdft8(C2<float>* v) {
  C2<float> e[4] = {v[0], v[2], v[4], v[6]};
  C2<float> o[4] = {v[1], v[3], v[5], v[7]};
  pdft4<INV>(e);
  pdft4<INV>(o);
  // w8 o1 and w8^3 o3 with w8 = exp(-+ i pi / 4)
  const C2<float> t1 = twc<8, INV>(o[1], 1), t3 = twc<8, INV>(o[3], 3);
  v[0] = padd(e[0], o[0]);
  v[4] = psub(e[0], o[0]);
  v[1] = padd(e[1], t1);
  v[5] = psub(e[1], t1);
  v[2] = add_rot<INV>(e[2], o[2]);
  v[6] = sub_rot<INV>(e[2], o[2]);
  v[3] = padd(e[3], t3);
  v[7] = psub(e[3], t3);
}

template <bool INV>
__device__ __forceinline__ void dft16(C2<float>* v) {
  C2<float> y[16];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    C2<float> a[4] = {v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]};
    pdft4<INV>(a);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) y[n1 * 4 + k2] = twc<16, INV>(a[k2], n1 * k2);
  }
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    C2<float> b[4] = {y[k2], y[4 + k2], y[8 + k2], y[12 + k2]};
    pdft4<INV>(b);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) v[k2 + 4 * k1] = b[k1];
  }
}

// Composite register DFT of size R = P * Q (Cooley-Tukey in registers):
// n = n1 + P n2, k = k2 + Q k1; twiddles exp(-+2 pi i n1 k2 / R) as rotations (twc).
template <int R> struct Split;
template <> struct Split<6> { static constexpr int P = 2, Q = 3; };
template <> struct Split<10> { static constexpr int P = 2, Q = 5; };
template <> struct Split<12> { static constexpr int P = 4, Q = 3; };
template <> struct Split<20> { static constexpr int P = 4, Q = 5; };
template <> struct Split<24> { static constexpr int P = 8, Q = 3; };

template <int R, bool INV>
__device__ __forceinline__ void dft_reg(C2<float>* v);

template <int R, bool INV>
__device__ __forceinline__ void dft_composite(C2<float>* v) {
  constexpr int P = Split<R>::P, Q = Split<R>::Q;
  C2<float> y[R];
#pragma unroll
  for (int n1 = 0; n1 < P; ++n1) {
    C2<float> a[Q];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) a[n2] = v[n1 + P * n2];
    dft_reg<Q, INV>(a);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) y[n1 * Q + k2] = twc<R, INV>(a[k2], (n1 * k2) % R);
  }
#pragma unroll
  for (int k2 = 0; k2 < Q; ++k2) {
    C2<float> b[P];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) b[n1] = y[n1 * Q + k2];
    dft_reg<P, INV>(b);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) v[k2 + Q * k1] = b[k1];
  }
}

template <int R, bool INV>
__device__ __forceinline__ void dft_reg(C2<float>* v) {
  if constexpr (R == 2) pdft2<INV>(v);
  else if constexpr (R == 3) pdft3<INV>(v);
  else if constexpr (R == 4) pdft4<INV>(v);
  else if constexpr (R == 5) pdft5<INV>(v);
  else if constexpr (R == 8) pdft8<INV>(v);
  else if constexpr (R == 16) dft16<INV>(v);
  else dft_composite<R, INV>(v);
}

// exchange slots: padded [R1][R2 + 1] rows
template <int R2>
struct XPad {
  C2<float>* p;
  __device__ __forceinline__ C2<float>& operator()(int n1, int k2) const { return p[n1 * (R2 + 1) + k2]; }
};
// Slot of k2 in row n1 of the exchange (n1, k2 < R2): a bijection on each row and on
// each column of slots, so that the row writes (fixed k2) and the column reads (fixed n1)
// of a line group both meet R2 distinct slots mod R2.  k2 XOR n1 for power-of-two R2 (one
// logic instruction with a compile-time k2 or n1), (k2 + n1) mod R2 otherwise.
template <int R2>
__device__ __forceinline__ int xskew(int n1, int k2) {
  if constexpr ((R2 & (R2 - 1)) == 0) {
    return k2 ^ n1;
  } else {
    int m = k2 + n1;
    if (m >= R2) m -= R2;
    return m;
  }
}
// exchange slots inside a strided line of L elements, skewed so that both the row
// writes and the column reads hit distinct banks
template <int R2>
struct XSkew {
  C2<float>* p;
  int s;
  __device__ __forceinline__ C2<float>& operator()(int n1, int k2) const {  // n1 < R2
    return p[s * (n1 * R2 + xskew<R2>(n1, k2))];
  }
};

// Twiddles w_L^(n1*k2) in a padded [R1][R2 + 1] table: a warp's threads (consecutive
// n1, one k2) then read distinct banks.  tw2 is filled by fill_tw2 from the table of
// w_L^m, m < L (n1 k2 < R1 R2 = L).
template <int L>
__host__ __device__ constexpr int tw2_size() { return RegPlan<L>::R1 * (RegPlan<L>::R2 + 1); }
template <int L>
__device__ __forceinline__ C2<float> tw2_entry(const C2<float>* __restrict__ tw, int i) {
  constexpr int R2 = RegPlan<L>::R2;
  const int n1 = i / (R2 + 1), k2 = i % (R2 + 1);
  return k2 < R2 ? tw[n1 * k2] : C2<float>{1.f, 0.f};
}
template <int L>
__device__ __forceinline__ void fill_tw2(C2<float>* tw2, const C2<float>* __restrict__ tw) {
  for (int i = threadIdx.x; i < tw2_size<L>(); i += blockDim.x) tw2[i] = tw2_entry<L>(tw, i);
}

// The inputs one thread of a line group holds: reg_load fills them, reg_fft_loaded
// transforms them (reg_fft does both; split, a caller can issue the loads of its first
// line before other setup work and its barrier).
template <int L>
struct RegLine {
  static constexpr int R1 = RegPlan<L>::R1, R2 = RegPlan<L>::R2, NT = reg_nt<L>();
  static constexpr int A = R1 / NT;
  C2<float> v[A][R2];
};
template <int L, class Ld>
__device__ __forceinline__ void reg_load(RegLine<L>& in, const Ld& ld, int t, bool active) {
  constexpr int R1 = RegPlan<L>::R1, R2 = RegPlan<L>::R2, NT = reg_nt<L>(), A = R1 / NT;
  if (active) {
#pragma unroll
    for (int a = 0; a < A; ++a)
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) in.v[a][n2] = ld(t + NT * a + R1 * n2);
  }
}

template <bool INV, int L, class Xch, class St>
__device__ __forceinline__ void reg_fft_loaded(RegLine<L>& in, const Xch& x, const St& st, const C2<float>* __restrict__ tw2,
                                               int t, bool active) {
  constexpr int R1 = RegPlan<L>::R1, R2 = RegPlan<L>::R2, NT = reg_nt<L>();
  constexpr int A = R1 / NT, B = (R2 + NT - 1) / NT;
  static_assert(R1 % NT == 0, "step 1 needs whole DFTs per thread");
  auto& v = in.v;
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
        x(n1, k2) = cmul_rn(v[a][k2], w);
      }
    }
  }
  __syncwarp();
  C2<float> u[B][R1];
  if (active) {
#pragma unroll
    for (int b = 0; b < B; ++b)
      if (R2 % NT == 0 || t + NT * b < R2) {
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) u[b][n1] = x(n1, t + NT * b);
      }
  }
  __syncwarp();
  if (active) {
#pragma unroll
    for (int b = 0; b < B; ++b)
      if (R2 % NT == 0 || t + NT * b < R2) {
        dft_reg<R1, INV>(u[b]);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) st(t + NT * b + R2 * k1, u[b][k1]);
      }
  }
  __syncwarp();
}

template <bool INV, int L, class Ld, class Xch, class St>
__device__ __forceinline__ void reg_fft(const Ld& ld, const Xch& x, const St& st, const C2<float>* __restrict__ tw2, int t,
                                        bool active) {
  RegLine<L> in;
  reg_load<L>(in, ld, t, active);
  reg_fft_loaded<INV, L>(in, x, st, tw2, t, active);
}

}  // namespace okmc
