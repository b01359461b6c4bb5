// Register-level DFTs and the in-CTA four-step transform used by every NLINV pass.
//
// A length-N transform (N = N1 * N2) is split the four-step way:
//   X[N2*k1 + k2] = sum_{n1} W_N1^{n1 k1} W_N^{n1 k2} sum_{n2} x[n1 + N1 n2] W_N2^{n2 k2},   W_R = exp(D 2 pi i / R)
// with D = -1 for the forward and +1 for the inverse transform.  One "lane" (a row or a column of a plane) is
// served by max(N1, N2) threads.  Two register layouts occur:
//   layout A(N1, N2): thread a < N1 holds elements a + N1*m, m < N2;
//   layout B(N1, N2): thread b < N2 holds elements b + N2*m, m < N1   (= layout A(N2, N1)).
// fft_AtoB takes layout A to layout B with one exchange through shared memory; a transform along the same axis
// that follows it uses the transposed split (N2, N1) and takes layout B back to layout A, so an inverse
// transform, a pointwise step and a forward transform need only two exchanges.
#pragma once
#include <cuda_runtime.h>
#include <utility>

namespace nlv {

// ---------------------------------------------------------------------------------------------- complex ----
// Complex sums and differences on the GPU use the paired FP32 instructions (add/sub .f32x2, one instruction for
// both parts, each part rounded as the scalar operation would be).
#if defined(__CUDA_ARCH__)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "add.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
#else
__host__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
#endif
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// i * a  and  -i * a
__host__ __device__ __forceinline__ float2 mul_i(float2 a) { return make_float2(-a.y, a.x); }
__host__ __device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }
// exp(D i pi/2) * a for D = +-1
template <int D> __host__ __device__ __forceinline__ float2 mul_di(float2 a) { return D > 0 ? mul_i(a) : mul_mi(a); }
// a + D i b and a - D i b in scalar form: the swap and the sign of D i b fold into the two additions
template <int D> __host__ __device__ __forceinline__ float2 cadd_di(float2 a, float2 b) {
  return D > 0 ? make_float2(a.x - b.y, a.y + b.x) : make_float2(a.x + b.y, a.y - b.x);
}
template <int D> __host__ __device__ __forceinline__ float2 csub_di(float2 a, float2 b) {
  return D > 0 ? make_float2(a.x + b.y, a.y - b.x) : make_float2(a.x - b.y, a.y + b.x);
}

// ------------------------------------------------------------------------------ compile-time helpers ----
template <class F, int... Is>
__host__ __device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
// Calls f(std::integral_constant<int, i>) for i = 0 .. N-1; every index is a compile-time constant.
template <int N, class F> __host__ __device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// sin and cos of 2 pi m / R in double, evaluated by the compiler: reduce to the first octant and sum the Taylor
// series there (|x| <= pi/4, 14 terms is far below double rounding).
constexpr double kPi = 3.14159265358979323846264338327950288;
__host__ __device__ constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 14; ++k) { term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0)); sum += term; }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 14; ++k) { term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k)); sum += term; }
  return sum;
}
// cos and sin of 2 pi t for t in [0, 1), reduced through the symmetries of the circle to [0, 1/8].
__host__ __device__ constexpr double cos2pi_oct(double t) {   // t in [0, 1/4]
  return (8.0 * t > 1.0) ? taylor_sin(2.0 * kPi * (0.25 - t)) : taylor_cos(2.0 * kPi * t);
}
__host__ __device__ constexpr double sin2pi_oct(double t) {   // t in [0, 1/4]
  return (8.0 * t > 1.0) ? taylor_cos(2.0 * kPi * (0.25 - t)) : taylor_sin(2.0 * kPi * t);
}
__host__ __device__ constexpr double cos2pi(double t) {
  if (t > 0.5) t = 1.0 - t;
  return (t > 0.25) ? -cos2pi_oct(0.5 - t) : cos2pi_oct(t);
}
__host__ __device__ constexpr double sin2pi(double t) {
  if (t > 0.5) return -sin2pi(1.0 - t);
  return (t > 0.25) ? sin2pi_oct(0.5 - t) : sin2pi_oct(t);
}
__host__ __device__ constexpr double unit_cos(long m, long R) { return cos2pi((double)(((m % R) + R) % R) / (double)R); }
__host__ __device__ constexpr double unit_sin(long m, long R) { return sin2pi((double)(((m % R) + R) % R) / (double)R); }

// a * exp(D 2 pi i M / R) with the factor known at compile time; exact for multiples of a quarter turn.
template <int R, int M, int D>
__host__ __device__ __forceinline__ float2 twiddle_c(float2 a) {
  constexpr int m = ((M % R) + R) % R;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (2 * m == R) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (4 * m == R) {
    return mul_di<D>(a);
  } else if constexpr (4 * m == 3 * R) {
    return mul_di<-D>(a);
  } else {
    constexpr float c = (float)unit_cos(m, R);
    constexpr float s = (float)(D * unit_sin(m, R));
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
  }
}

// ------------------------------------------------------------------------------------- register DFTs ----
// In-place DFT of R values, natural order in and out: a[k] <- sum_n a[n] exp(D 2 pi i n k / R).
template <int R, int D> struct RegDFT;

template <int D> struct RegDFT<1, D> {
  __host__ __device__ __forceinline__ static void run(float2*) {}
};

template <int D> struct RegDFT<2, D> {
  __host__ __device__ __forceinline__ static void run(float2* a) {
    float2 t = a[1];
    a[1] = csub(a[0], t);
    a[0] = cadd(a[0], t);
  }
};

template <int D> struct RegDFT<3, D> {
  __host__ __device__ __forceinline__ static void run(float2* a) {
    constexpr float h = 0.86602540378443864676f;      // sin(2 pi / 3)
    float2 s = cadd(a[1], a[2]);
    float2 d = csub(a[1], a[2]);
    float2 m = make_float2(fmaf(-0.5f, s.x, a[0].x), fmaf(-0.5f, s.y, a[0].y));
    // a1 = m + D i h d, a2 = m - D i h d, as fused multiply-adds
    constexpr float dh = D > 0 ? h : -h;
    a[0] = cadd(a[0], s);
    a[1] = make_float2(fmaf(-dh, d.y, m.x), fmaf(dh, d.x, m.y));
    a[2] = make_float2(fmaf(dh, d.y, m.x), fmaf(-dh, d.x, m.y));
  }
};

template <int D> struct RegDFT<4, D> {
  __host__ __device__ __forceinline__ static void run(float2* a) {
    float2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
    float2 s13 = cadd(a[1], a[3]), d13 = csub(a[1], a[3]);
    a[0] = cadd(s02, s13);
    a[2] = csub(s02, s13);
    a[1] = cadd_di<D>(d02, d13);
    a[3] = csub_di<D>(d02, d13);
  }
};

template <int D> struct RegDFT<5, D> {
  __host__ __device__ __forceinline__ static void run(float2* a) {
    constexpr float c1 = (float)unit_cos(1, 5), c2 = (float)unit_cos(2, 5);
    constexpr float s1 = (float)unit_sin(1, 5), s2 = (float)unit_sin(2, 5);
    float2 b1 = cadd(a[1], a[4]), d1 = csub(a[1], a[4]);
    float2 b2 = cadd(a[2], a[3]), d2 = csub(a[2], a[3]);
    float2 e1 = make_float2(a[0].x + c1 * b1.x + c2 * b2.x, a[0].y + c1 * b1.y + c2 * b2.y);
    float2 e2 = make_float2(a[0].x + c2 * b1.x + c1 * b2.x, a[0].y + c2 * b1.y + c1 * b2.y);
    float2 f1 = make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
    float2 f2 = make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
    a[0] = make_float2(a[0].x + b1.x + b2.x, a[0].y + b1.y + b2.y);
    a[1] = cadd_di<D>(e1, f1);
    a[4] = csub_di<D>(e1, f1);
    a[2] = cadd_di<D>(e2, f2);
    a[3] = csub_di<D>(e2, f2);
  }
};

__host__ __device__ constexpr int first_factor(int R) {
  return (R % 4 == 0 && R != 4) ? 4 : (R % 2 == 0 && R != 2) ? 2 : (R % 3 == 0 && R != 3) ? 3
       : (R % 5 == 0 && R != 5) ? 5 : R;
}

// Composite sizes: the same four-step split, entirely in registers (R = Q1 * Q2, Q1 the leading factor).
template <int R, int D> struct RegDFT {
  static constexpr int Q1 = first_factor(R);
  static constexpr int Q2 = R / Q1;
  static_assert(Q1 * Q2 == R && Q1 > 1 && Q2 > 1, "register DFT size must factor into 2, 3, 4 and 5");
  __host__ __device__ __forceinline__ static void run(float2* a) {
    float2 t[R];
    static_for<Q1>([&](auto n1c) {
      constexpr int n1 = decltype(n1c)::value;
      float2 b[Q2];
      static_for<Q2>([&](auto n2c) { constexpr int n2 = decltype(n2c)::value; b[n2] = a[n1 + Q1 * n2]; });
      RegDFT<Q2, D>::run(b);
      static_for<Q2>([&](auto k2c) {
        constexpr int k2 = decltype(k2c)::value;
        t[n1 * Q2 + k2] = twiddle_c<R, n1 * k2, D>(b[k2]);
      });
    });
    static_for<Q2>([&](auto k2c) {
      constexpr int k2 = decltype(k2c)::value;
      float2 b[Q1];
      static_for<Q1>([&](auto n1c) { constexpr int n1 = decltype(n1c)::value; b[n1] = t[n1 * Q2 + k2]; });
      RegDFT<Q1, D>::run(b);
      static_for<Q1>([&](auto k1c) { constexpr int k1 = decltype(k1c)::value; a[Q2 * k1 + k2] = b[k1]; });
    });
  }
};

// ---------------------------------------------------------------------------------- in-CTA transform ----
template <int A, int B> struct Split {
  static constexpr int N1 = A, N2 = B, N = A * B;
  static constexpr int TL = A > B ? A : B;       // threads per lane
  static constexpr int E = TL;                   // register slots per thread
  // shared floats2 per lane for one exchange in either direction (row pitch N1+1 or N2+1, odd for even sizes)
  static constexpr int SM_AB = N2 * (N1 + 1);
  static constexpr int SM_BA = N1 * (N2 + 1);
  static constexpr int SM_LANE = (SM_AB > SM_BA ? SM_AB : SM_BA);
  // lane stride for passes whose adjacent threads belong to adjacent lanes (column passes): padded to 2 mod 16
  // float2 so that 8 lanes x 2 indices of a half-warp fall on distinct 8-byte banks
  static constexpr int SM_LANE_COL = SM_LANE + ((2 - SM_LANE % 16) + 16) % 16;
};

// Radix-16 register DFTs stay on the CUDA cores unless a tensor-core engine (tc_dft.cuh) is passed in.
struct NoTc {
  static constexpr bool enabled = false;
  template <int D, int E>
  __device__ __forceinline__ void dft16(float2 (&)[E], bool) {}
};

// Layout A(P1, P2) -> layout B(P1, P2) for one lane of P1*P2 points.
//   v      register slots of this thread (v[0..P2) valid on entry if idx < P1; v[0..P1) valid on exit if idx < P2)
//   sm     this lane's shared-memory exchange area (>= P2*(P1+1) float2)
//   tw     table tw[k2*P1 + a] = exp(-2 pi i a k2 / (P1 P2)) (forward sign; conjugated for D = +1), in shared
//          memory
// Contains two __syncthreads(): every thread of the CTA must call it.
// General form: the threads of the two steps may be mapped differently onto the lanes (a lane's exchange area is
// the same in both).  Step 1 runs on the threads with in_ok (index in_idx < P1 of the lane whose area is sm_in),
// step 3 on those with out_ok (index out_idx < P2, area sm_out).
// tc: with an enabled tensor-core engine, a radix-16 register DFT (step 1 when P2 = 16, step 3 when P1 = 16) runs
// as one block-wide tensor-core contraction instead (every thread takes part; threads without data pass zeros).
// TRAIL = false drops the closing barrier (CUDA-core stages only): for the last exchange of a pass, when every
// later write to the exchange area comes after another block-wide barrier (the next round's or work item's).
template <int P1, int P2, int D, int E, class TC = NoTc, bool TRAIL = true>
__device__ __forceinline__ void fft_AtoB2(float2 (&v)[E], float2* sm_in, int in_idx, bool in_ok, float2* sm_out,
                                          int out_idx, bool out_ok, const float2* tw, TC* tc = nullptr) {
  constexpr int S = P1 + 1;
  constexpr bool tc1 = TC::enabled && P2 == 16;
  constexpr bool tc3 = TC::enabled && P1 == 16;
  if constexpr (tc1) tc->template dft16<D>(v, in_ok);
  if (in_ok) {
    if constexpr (!tc1) RegDFT<P2, D>::run(v);
    static_for<P2>([&](auto kc) {
      constexpr int k2 = decltype(kc)::value;
      float2 w = tw[k2 * P1 + in_idx];
      if (D > 0) w.y = -w.y;
      sm_in[k2 * S + in_idx] = (k2 == 0) ? v[k2] : cmul(v[k2], w);
    });
  }
  __syncthreads();
  if (out_ok) {
    static_for<P1>([&](auto nc) { constexpr int n1 = decltype(nc)::value; v[n1] = sm_out[out_idx * S + n1]; });
    if constexpr (!tc3) RegDFT<P1, D>::run(v);
  }
  if constexpr (tc3) tc->template dft16<D>(v, out_ok);
  if constexpr (TRAIL || TC::enabled) __syncthreads();
}

template <int P1, int P2, int D, bool TRAIL = true, int E, class TC = NoTc>
__device__ __forceinline__ void fft_AtoB(float2 (&v)[E], float2* sm, const float2* tw, int idx, TC* tc = nullptr) {
  fft_AtoB2<P1, P2, D, E, TC, TRAIL>(v, sm, idx, idx < P1, sm, idx, idx < P2, tw, tc);
}

}  // namespace nlv
