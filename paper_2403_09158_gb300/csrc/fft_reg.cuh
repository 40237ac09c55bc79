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
template <bool INV> __device__ __forceinline__ void pdft8(C2<float>* v) {
  const float h = 0.70710678118654752440f;  // sqrt(1/2)
  C2<float> e[4] = {v[0], v[2], v[4], v[6]};
  C2<float> o[4] = {v[1], v[3], v[5], v[7]};
  pdft4<INV>(e);
  pdft4<INV>(o);
  // w8 o1 = h * t1 and w8^3 o3 = h * t3 with w8 = exp(-+ i pi / 4)
  const C2<float> t1 = INV ? C2<float>{o[1].x - o[1].y, o[1].x + o[1].y} : C2<float>{o[1].x + o[1].y, o[1].y - o[1].x};
  const C2<float> t3 = INV ? C2<float>{-o[3].x - o[3].y, o[3].x - o[3].y} : C2<float>{o[3].y - o[3].x, -o[3].x - o[3].y};
  v[0] = padd(e[0], o[0]);
  v[4] = psub(e[0], o[0]);
  v[1] = pfma(h, t1, e[1]);
  v[5] = pfma(-h, t1, e[1]);
  v[2] = add_rot<INV>(e[2], o[2]);
  v[6] = sub_rot<INV>(e[2], o[2]);
  v[3] = pfma(h, t3, e[3]);
  v[7] = pfma(-h, t3, e[3]);
}

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
  return cmul_rn(v, C2<float>{c, s});
}

template <bool INV>
__device__ __forceinline__ void dft16(C2<float>* v) {
  C2<float> y[16];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    C2<float> a[4] = {v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]};
    pdft4<INV>(a);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) y[n1 * 4 + k2] = tw16<INV>(a[k2], n1 * k2);
  }
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    C2<float> b[4] = {y[k2], y[4 + k2], y[8 + k2], y[12 + k2]};
    pdft4<INV>(b);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) v[k2 + 4 * k1] = b[k1];
  }
}

template <int N> __device__ __forceinline__ float cosN(int e);
template <int N> __device__ __forceinline__ float sinN(int e);
// cos and sin of 2 pi e / N for the composite register DFTs (e = 0..N-1)
template <> __device__ __forceinline__ float cosN<6>(int e) {
  switch (e) {
    case 0: return 1.0f;
    case 1: return 0.5f;
    case 2: return -0.5f;
    case 3: return -1.0f;
    case 4: return -0.5f;
    default: return 0.5f;
  }
}
template <> __device__ __forceinline__ float sinN<6>(int e) {
  switch (e) {
    case 0: return 0.0f;
    case 1: return 0.8660254037844386f;
    case 2: return 0.86602540378443871f;
    case 3: return 0.0f;
    case 4: return -0.86602540378443837f;
    default: return -0.8660254037844386f;
  }
}
template <> __device__ __forceinline__ float cosN<10>(int e) {
  switch (e) {
    case 0: return 1.0f;
    case 1: return 0.80901699437494745f;
    case 2: return 0.30901699437494745f;
    case 3: return -0.30901699437494734f;
    case 4: return -0.80901699437494734f;
    case 5: return -1.0f;
    case 6: return -0.80901699437494756f;
    case 7: return -0.30901699437494756f;
    case 8: return 0.30901699437494723f;
    default: return 0.80901699437494734f;
  }
}
template <> __device__ __forceinline__ float sinN<10>(int e) {
  switch (e) {
    case 0: return 0.0f;
    case 1: return 0.58778525229247314f;
    case 2: return 0.95105651629515353f;
    case 3: return 0.95105651629515364f;
    case 4: return 0.58778525229247325f;
    case 5: return 0.0f;
    case 6: return -0.58778525229247303f;
    case 7: return -0.95105651629515353f;
    case 8: return -0.95105651629515364f;
    default: return -0.58778525229247336f;
  }
}
template <> __device__ __forceinline__ float cosN<12>(int e) {
  switch (e) {
    case 0: return 1.0f;
    case 1: return 0.86602540378443871f;
    case 2: return 0.5f;
    case 3: return 0.0f;
    case 4: return -0.5f;
    case 5: return -0.86602540378443871f;
    case 6: return -1.0f;
    case 7: return -0.86602540378443882f;
    case 8: return -0.5f;
    case 9: return 0.0f;
    case 10: return 0.5f;
    default: return 0.86602540378443837f;
  }
}
template <> __device__ __forceinline__ float sinN<12>(int e) {
  switch (e) {
    case 0: return 0.0f;
    case 1: return 0.5f;
    case 2: return 0.8660254037844386f;
    case 3: return 1.0f;
    case 4: return 0.86602540378443871f;
    case 5: return 0.5f;
    case 6: return 0.0f;
    case 7: return -0.5f;
    case 8: return -0.86602540378443837f;
    case 9: return -1.0f;
    case 10: return -0.8660254037844386f;
    default: return -0.5f;
  }
}
template <> __device__ __forceinline__ float cosN<20>(int e) {
  switch (e) {
    case 0: return 1.0f;
    case 1: return 0.95105651629515353f;
    case 2: return 0.80901699437494745f;
    case 3: return 0.58778525229247314f;
    case 4: return 0.30901699437494745f;
    case 5: return 0.0f;
    case 6: return -0.30901699437494734f;
    case 7: return -0.58778525229247303f;
    case 8: return -0.80901699437494734f;
    case 9: return -0.95105651629515353f;
    case 10: return -1.0f;
    case 11: return -0.95105651629515375f;
    case 12: return -0.80901699437494756f;
    case 13: return -0.58778525229247325f;
    case 14: return -0.30901699437494756f;
    case 15: return 0.0f;
    case 16: return 0.30901699437494723f;
    case 17: return 0.58778525229247292f;
    case 18: return 0.80901699437494734f;
    default: return 0.95105651629515353f;
  }
}
template <> __device__ __forceinline__ float sinN<20>(int e) {
  switch (e) {
    case 0: return 0.0f;
    case 1: return 0.3090169943749474f;
    case 2: return 0.58778525229247314f;
    case 3: return 0.80901699437494745f;
    case 4: return 0.95105651629515353f;
    case 5: return 1.0f;
    case 6: return 0.95105651629515364f;
    case 7: return 0.80901699437494745f;
    case 8: return 0.58778525229247325f;
    case 9: return 0.30901699437494751f;
    case 10: return 0.0f;
    case 11: return -0.3090169943749469f;
    case 12: return -0.58778525229247303f;
    case 13: return -0.80901699437494734f;
    case 14: return -0.95105651629515353f;
    case 15: return -1.0f;
    case 16: return -0.95105651629515364f;
    case 17: return -0.80901699437494756f;
    case 18: return -0.58778525229247336f;
    default: return -0.30901699437494762f;
  }
}
template <> __device__ __forceinline__ float cosN<24>(int e) {
  switch (e) {
    case 0: return 1.0f;
    case 1: return 0.96592582628906831f;
    case 2: return 0.86602540378443871f;
    case 3: return 0.70710678118654757f;
    case 4: return 0.5f;
    case 5: return 0.25881904510252074f;
    case 6: return 0.0f;
    case 7: return -0.25881904510252063f;
    case 8: return -0.5f;
    case 9: return -0.70710678118654746f;
    case 10: return -0.86602540378443871f;
    case 11: return -0.9659258262890682f;
    case 12: return -1.0f;
    case 13: return -0.96592582628906831f;
    case 14: return -0.86602540378443882f;
    case 15: return -0.70710678118654791f;
    case 16: return -0.5f;
    case 17: return -0.25881904510252063f;
    case 18: return 0.0f;
    case 19: return 0.2588190451025203f;
    case 20: return 0.5f;
    case 21: return 0.70710678118654735f;
    case 22: return 0.86602540378443837f;
    default: return 0.96592582628906809f;
  }
}
template <> __device__ __forceinline__ float sinN<24>(int e) {
  switch (e) {
    case 0: return 0.0f;
    case 1: return 0.25881904510252074f;
    case 2: return 0.5f;
    case 3: return 0.70710678118654746f;
    case 4: return 0.8660254037844386f;
    case 5: return 0.96592582628906831f;
    case 6: return 1.0f;
    case 7: return 0.96592582628906831f;
    case 8: return 0.86602540378443871f;
    case 9: return 0.70710678118654757f;
    case 10: return 0.5f;
    case 11: return 0.25881904510252102f;
    case 12: return 0.0f;
    case 13: return -0.25881904510252079f;
    case 14: return -0.5f;
    case 15: return -0.70710678118654713f;
    case 16: return -0.86602540378443837f;
    case 17: return -0.96592582628906831f;
    case 18: return -1.0f;
    case 19: return -0.96592582628906842f;
    case 20: return -0.8660254037844386f;
    case 21: return -0.70710678118654768f;
    case 22: return -0.5f;
    default: return -0.25881904510252157f;
  }
}

// Composite register DFT of size R = P * Q (Cooley-Tukey in registers):
// n = n1 + P n2, k = k2 + Q k1; twiddles exp(-+2 pi i n1 k2 / R) from the tables above.
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
    for (int k2 = 0; k2 < Q; ++k2) {
      const int e = (n1 * k2) % R;
      if (e == 0) {
        y[n1 * Q + k2] = a[k2];
      } else {
        const float c = cosN<R>(e), s = INV ? sinN<R>(e) : -sinN<R>(e);
        y[n1 * Q + k2] = cmul_rn(a[k2], C2<float>{c, s});
      }
    }
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
// exchange slots inside a strided line of L elements, skewed so that both the row
// writes and the column reads hit distinct banks
template <int R2>
struct XSkew {
  C2<float>* p;
  int s;
  __device__ __forceinline__ C2<float>& operator()(int n1, int k2) const {  // n1 < R2
    int m = k2 + n1;
    if (m >= R2) m -= R2;
    return p[s * (n1 * R2 + m)];
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
