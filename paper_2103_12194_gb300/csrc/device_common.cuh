// Device helpers shared by the kernels of libslpic: Philox4x32-10, the
// uniform map, the speed limiter and the kinematic building blocks.
//
// The whole library is compiled with -fmad=false and IEEE division and square
// root, so every expression below is evaluated with one rounding per
// operation, in the order written; a fused multiply-add appears only where
// the source asks for one (mad, __fmaf_rn).
#pragma once

#include <cuda/atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include "slpic_internal.h"

namespace slpic {

// Programmatic dependent launch between the kernels of a step: each kernel
// lets the next one be scheduled at once (its CTAs take SMs as this grid's
// CTAs leave) and waits, before its first read of global memory, until the
// previous grid has completed and its writes are visible.  Launched without
// the attribute, the wait returns at once.
__device__ __forceinline__ void step_kernel_entry() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launch a step kernel with programmatic stream serialization (see
// step_kernel_entry); errors surface through cudaGetLastError like <<<>>>.
template <typename... P, typename... A>
inline void launch_step_kernel(void (*kernel)(P...), int grid, int threads, size_t smem,
                               cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned int)grid);
  cfg.blockDim = dim3((unsigned int)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  (void)cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 32x32 -> 64-bit products of counter words 0 and 2 with the round
// multipliers, the high halves mixed with the other words and the round key;
// the key advances by the Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    // one 32x32 -> 64-bit product each (a single wide multiply instruction)
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Philox2x32-10 (same publication): one 32x32 -> 64-bit product per round,
// the high half mixed with the other counter word and the round key; the key
// advances by the Weyl increment between rounds.  Used for the one draw every
// electron makes every step (the null-collision test), where it costs half of
// Philox4x32-10.
__device__ __forceinline__ uint2 philox2x32_10(uint2 c, uint32_t k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) k += 0x9E3779B9u;
    const unsigned long long p = (unsigned long long)0xD256D193u * c.x;
    c = make_uint2((uint32_t)(p >> 32) ^ c.y ^ k, (uint32_t)p);
  }
  return c;
}

// 32 random bits -> (floor(x / 2^9) + 1/2) 2^-23, exactly representable.
__device__ __forceinline__ float uniform01(uint32_t x) {
  return (__uint2float_rn(x >> 9) + 0.5f) * 1.1920928955078125e-07f;
}

// The step's constants and node field in the arithmetic type R.
template <typename R>
__device__ __forceinline__ const StepConsts<R>& consts(const InstDev& P);
template <>
__device__ __forceinline__ const StepConsts<float>& consts<float>(const InstDev& P) {
  return P.c32;
}
template <>
__device__ __forceinline__ const StepConsts<double>& consts<double>(const InstDev& P) {
  return P.c64;
}
template <typename R>
__device__ __forceinline__ const R* node_field(const InstDev& P);
template <>
__device__ __forceinline__ const float* node_field<float>(const InstDev& P) {
  return P.E32;
}
template <>
__device__ __forceinline__ const double* node_field<double>(const InstDev& P) {
  return P.E64;
}

// Elementary functions by precision (the library's own float and double
// versions; nothing here is fused or approximated).
__device__ __forceinline__ float r_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double r_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float r_floor(float x) { return floorf(x); }
__device__ __forceinline__ double r_floor(double x) { return floor(x); }
__device__ __forceinline__ float r_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double r_min(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float r_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double r_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float r_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double r_abs(double x) { return fabs(x); }
__device__ __forceinline__ float r_log(float x) { return logf(x); }
__device__ __forceinline__ double r_log(double x) { return log(x); }
__device__ __forceinline__ float r_exp(float x) { return expf(x); }
__device__ __forceinline__ double r_exp(double x) { return exp(x); }
__device__ __forceinline__ float r_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double r_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float r_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double r_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float r_cos(float x) { return cosf(x); }
__device__ __forceinline__ double r_cos(double x) { return cos(x); }
__device__ __forceinline__ float r_sin(float x) { return sinf(x); }
__device__ __forceinline__ double r_sin(double x) { return sin(x); }
__device__ __forceinline__ float r_pow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double r_pow(double x, double y) { return pow(x, y); }

// Largest value of R below 1.
template <typename R>
__device__ __forceinline__ R nextafter_below_one();
template <>
__device__ __forceinline__ float nextafter_below_one<float>() {
  return __int_as_float(0x3F7FFFFF);
}
template <>
__device__ __forceinline__ double nextafter_below_one<double>() {
  return __longlong_as_double(0x3FEFFFFFFFFFFFFFll);
}

// The same uniform in R (exact in both types).
template <typename R>
__device__ __forceinline__ R uniform01r(uint32_t x) {
  return (R)uniform01(x);
}

template <typename R>
__device__ __forceinline__ void uniform4(uint4 r, R u[4]) {
  u[0] = uniform01r<R>(r.x);
  u[1] = uniform01r<R>(r.y);
  u[2] = uniform01r<R>(r.z);
  u[3] = uniform01r<R>(r.w);
}

// beta(v) = min(1, v_lim / v), Eq. betaAbrupt; v_lim = +inf gives 1.  Equal,
// bit for bit, to (v > v_lim ? v_lim / v : 1): when v <= v_lim the rounded
// quotient is >= 1 (rounding is monotone), and v = 0 gives +inf.
template <typename R>
__device__ __forceinline__ R beta_of(R v, R vlim) {
  return r_min((R)1, vlim / v);
}

// Multiply-add in the marker type: fused (one rounding) in float, where the
// kick spends its time; written out in double, the plain FP64 form.
__device__ __forceinline__ float mad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return a * b + c; }

// Natural logarithm of a positive normal float by Tang's table-driven method
// (P. T. P. Tang, "Table-driven implementation of the logarithm function in
// IEEE floating-point arithmetic", ACM TOMS 16, 1990), from IEEE operations
// and one table read, with no division:
//  - y = 2^k m with m in [0x3F350000, 0x3FB50000) as bit patterns
//    (about [0.707, 1.414)); the top 6 bits of m's offset from the lower end
//    pick interval j, whose centre c_j is the float at bit pattern
//    0x3F350000 + 2^17 j + 2^16 (c_37 = 1 exactly);
//  - kLogTab[j] = {r_j, n_j} with r_j = 1 / c_j rounded to float and n_j =
//    -log(r_j) rounded to nearest float (r_37 = 1, n_37 = 0);
//  - f = m r_j - 1 in one rounding (|f| < 2^-7), log(1 + f) by its Taylor
//    series to f^4 (the next term is below 2^-28 of the sum), and
//    log y = k log 2 + n_j + log(1 + f), with log 2 split in a 15-bit head
//    and a tail so that the product keeps its precision.
// In double the library's log is used.
__device__ const float2 kLogTab[64] = {
    {1.4065934e+00f, -3.411708e-01f}, {1.3913044e+00f, -3.302417e-01f}, {1.3763441e+00f, -3.1943077e-01f}, {1.3617021e+00f, -3.0873546e-01f},
    {1.3473685e+00f, -2.981534e-01f}, {1.3333334e+00f, -2.8768212e-01f}, {1.3195876e+00f, -2.7731925e-01f}, {1.3061224e+00f, -2.6706275e-01f},
    {1.2929293e+00f, -2.569104e-01f}, {1.28e+00f, -2.4686006e-01f}, {1.2673267e+00f, -2.3690973e-01f}, {1.254902e+00f, -2.2705749e-01f},
    {1.2427185e+00f, -2.1730128e-01f}, {1.2307693e+00f, -2.076394e-01f}, {1.2190477e+00f, -1.9806994e-01f}, {1.2075472e+00f, -1.8859118e-01f},
    {1.1962616e+00f, -1.792014e-01f}, {1.1851852e+00f, -1.6989905e-01f}, {1.1743119e+00f, -1.6068234e-01f}, {1.1636363e+00f, -1.5154986e-01f},
    {1.1531532e+00f, -1.4250009e-01f}, {1.1428572e+00f, -1.3353144e-01f}, {1.1327434e+00f, -1.2464244e-01f}, {1.122807e+00f, -1.1583182e-01f},
    {1.1130434e+00f, -1.0709809e-01f}, {1.1034483e+00f, -9.8440066e-02f}, {1.0940171e+00f, -8.985638e-02f}, {1.0847458e+00f, -8.134564e-02f},
    {1.0756303e+00f, -7.290682e-02f}, {1.0666667e+00f, -6.4538576e-02f}, {1.0578512e+00f, -5.6239676e-02f}, {1.0491803e+00f, -4.8009165e-02f},
    {1.0406504e+00f, -3.9845873e-02f}, {1.032258e+00f, -3.1748667e-02f}, {1.024e+00f, -2.3716575e-02f}, {1.0158731e+00f, -1.5748415e-02f},
    {1.007874e+00f, -7.843174e-03f}, {1.e+00f, 0.e+00f}, {9.846154e-01f, 1.5504186e-02f}, {9.69697e-01f, 3.0771628e-02f},
    {9.5522386e-01f, 4.580956e-02f}, {9.411765e-01f, 6.0624618e-02f}, {9.2753625e-01f, 7.52234e-02f}, {9.142857e-01f, 8.9612156e-02f},
    {9.0140843e-01f, 1.0379681e-01f}, {8.888889e-01f, 1.17783025e-01f}, {8.767123e-01f, 1.3157636e-01f}, {8.648649e-01f, 1.4518198e-01f},
    {8.5333335e-01f, 1.5860501e-01f}, {8.4210527e-01f, 1.7185025e-01f}, {8.3116883e-01f, 1.8492234e-01f}, {8.2051283e-01f, 1.9782573e-01f},
    {8.101266e-01f, 2.1056475e-01f}, {8.e-01f, 2.2314353e-01f}, {7.9012346e-01f, 2.3556606e-01f}, {7.804878e-01f, 2.478362e-01f},
    {7.710843e-01f, 2.5995755e-01f}, {7.619048e-01f, 2.719337e-01f}, {7.529412e-01f, 2.8376815e-01f}, {7.4418604e-01f, 2.9546422e-01f},
    {7.356322e-01f, 3.0702505e-01f}, {7.2727275e-01f, 3.184537e-01f}, {7.1910113e-01f, 3.2975328e-01f}, {7.111111e-01f, 3.4092656e-01f},
};
__device__ __forceinline__ float r_logk(float y) {
  const int ix = (int)__float_as_uint(y) - 0x3F350000;
  const int k = ix >> 23;
  const uint32_t mb = (uint32_t)ix & 0x7FFFFFu;
  const float m = __uint_as_float(mb + 0x3F350000u);
  const float2 t = __ldg(&kLogTab[mb >> 17]);
  const float f = __fmaf_rn(m, t.x, -1.0f);
  float q = __fmaf_rn(f, -0.25f, 1.0f / 3.0f);
  q = __fmaf_rn(f, q, -0.5f);
  const float lp = __fmaf_rn(f * f, q, f);
  const float kf = (float)k;
  return __fmaf_rn(kf, 0.693145751953125f, __fmaf_rn(kf, 1.428606765330187e-06f, t.y + lp));
}
__device__ __forceinline__ double r_logk(double y) { return log(y); }

// Halley steps of the kick stop once a step is below this fraction of the
// speed; the error left is then about its cube.
template <typename R>
__device__ __forceinline__ R kick_tol();
template <>
__device__ __forceinline__ float kick_tol<float>() {
  return 0.00390625f;  // 2^-8
}
template <>
__device__ __forceinline__ double kick_tol<double>() {
  return 3.814697265625e-06;  // 2^-18
}

// Speed-limited kick over one step of a species with a finite limit L
// (Eq. slpicEOMv: dv_x/dt = beta(|v|) q E_x / m with E_x held at its gathered
// value, v_y and v_z unchanged), for the N slots a lane advances.  A is the
// unlimited velocity increment q E_x dt / m; vx is replaced by the new v_x.
//  - Below the limit at both ends of the step: the leapfrog kick v_x + A.
//  - Otherwise the exact solution of the equation over the step.  In the
//    time tau = integral of beta dt the motion is unlimited,
//    v_x = v_x0 + (A / dt) tau, and dt = integral of max(1, |v| / L) dtau.
//    With w = v_x sign(A) the speed along the force and p2 = v_y^2 + v_z^2,
//    the step ends where the integral of max(L, sqrt(w^2 + p2)) dw from w0
//    reaches W = L |A|.  Along the force the path has up to three parts:
//    limited and slowing (w < -q), unlimited (|w| <= q, q^2 = L^2 - p2) and
//    limited and speeding up (w > q); the end lies in the first part whose
//    cost exhausts W.
//  - In a limited part the end speed m >= 0 solves D(m0, m) = T, where
//    D(a, b) = integral from a to b of sqrt(x^2 + p2) dx
//            = [b s_b - a s_a + p2 log((b + s_b) / (a + s_a))] / 2
//    and T = +W (speeding up) or -W (slowing down): a third-order series
//    guess in X = T / s0^2 (beyond |X| = 1/2, sqrt(m0^2 + 2 T)), then Halley
//    steps (D' = s, D'' = m / s) kept inside a bracket until a step is below
//    kick_tol of the speed.
// The slots take their Halley steps together, one step of every unfinished
// slot per round, so that their dependency chains interleave; each slot's
// arithmetic is that of a kick computed alone.  Only + - * / sqrt (and fused
// multiply-adds in float) are used, so an FP32 restatement reproduces it bit
// for bit.
template <typename R, int N>
__device__ __forceinline__ void limited_kick_n(R (&vx)[N], const R (&vy)[N], const R (&vz)[N],
                                               const R (&A)[N], R L) {
  const R L2 = L * L;
  const R tau = kick_tol<R>();
  R m[N], m0[N], T[N], lo[N], hi[N], p2[N], ih0[N], hm0s0[N], gs[N];
  bool act[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    act[j] = false;
    p2[j] = mad(vy[j], vy[j], vz[j] * vz[j]);
    const R sp2 = mad(vx[j], vx[j], p2[j]);
    const R vt = vx[j] + A[j];
    if (sp2 <= L2 && mad(vt, vt, p2[j]) <= L2) {
      vx[j] = vt;
      continue;
    }
    if (!(A[j] != (R)0)) continue;
    const R g = A[j] > (R)0 ? (R)1 : (R)-1;
    const R W = L * (g * A[j]);
    const R w = g * vx[j];
    // the unlimited zone |w| <= q (empty when p2 >= L2)
    const R q = r_sqrt(r_max(L2 - p2[j], (R)0));
    const R s0 = r_sqrt(sp2);
    const R a0 = -w;
    // Limited and slowing down (w < -q): reaching the zone (or the axis,
    // when p2 >= L2) costs C1 = D(q, |w|) >= L (|w| - q).  C1 is formed only
    // by the lanes whose budget exceeds that lower bound (a warp with none
    // skips it); the others stay in the slowing part, or start elsewhere.
    const bool regI = w < -q;
    const bool near = regI && !(W <= L * (a0 - q));
    R C1 = (R)0;
    if (near) {
      const R sq = q > (R)0 ? L : r_sqrt(p2[j]);
      C1 = (R)0.5 * (a0 * s0 - q * sq);
      if (p2[j] > (R)0) C1 = mad((R)0.5 * p2[j], r_logk((a0 + s0) / (q + sq)), C1);
    }
    const bool stay = regI && (!near || W < C1);
    // otherwise the limited part that speeds up starts at wf with budget Wf
    R wf = regI ? -q : w;
    R Wf = regI ? W - C1 : W;
    R s0f = s0;
    if (!stay && wf < q) {
      // the unlimited zone (rare in a warp): the step may end inside it
      const R reach = L * (q - wf);
      if (Wf <= reach) {
        vx[j] = g * (wf + Wf / L);
        continue;
      }
      Wf = Wf - reach;
      wf = q;
    }
    if (!stay && wf != w) s0f = r_sqrt(mad(wf, wf, p2[j]));
    m0[j] = stay ? a0 : wf;
    T[j] = stay ? -W : Wf;
    lo[j] = stay ? q : wf;
    gs[j] = stay ? -g : g;
    const R s0s = stay ? s0 : s0f;
    // the solve's constants and its starting guess
    const R h0 = m0[j] + s0s;
    const R rr = (R)1 / (s0s * h0);
    const R is0 = h0 * rr;
    ih0[j] = s0s * rr;
    hi[j] = stay ? a0 : mad(T[j], is0, m0[j]);  // speeding up: s >= s0 along the way
    const R X = (T[j] * is0) * is0;
    const R c0 = m0[j] * is0;
    R mg;
    if (r_abs(X) <= (R)0.5) {
      const R c3 = mad((R)4 * c0, c0, (R)-1) * (R)(1.0 / 6.0);
      const R zh = X * mad(X, mad(X, c3, (R)-0.5 * c0), (R)1);
      mg = mad(s0s, zh, m0[j]);
    } else {
      mg = r_sqrt(r_max((R)0, mad(m0[j], m0[j], T[j] + T[j])));
    }
    m[j] = r_min(r_max(mg, lo[j]), hi[j]);
    hm0s0[j] = (R)0.5 * (m0[j] * s0s);
    act[j] = true;
  }
  bool any = false;
#pragma unroll
  for (int j = 0; j < N; ++j) any |= act[j];
  for (int it = 0; it < 24 && any; ++it) {
    any = false;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      if (!act[j]) continue;
      const R s = r_sqrt(mad(m[j], m[j], p2[j]));
      const R lg = p2[j] > (R)0 ? r_logk((m[j] + s) * ih0[j]) : (R)0;
      const R F = mad((R)0.5 * p2[j], lg, mad((R)0.5 * m[j], s, -hm0s0[j])) - T[j];
      if (F > (R)0) hi[j] = m[j];
      else lo[j] = m[j];
      const R s2 = s * s;
      const R dm = ((F + F) * s2) / mad(s2 + s2, s, -(F * m[j]));
      R mn = m[j] - dm;
      if (!(mn >= lo[j] && mn <= hi[j])) mn = (R)0.5 * (lo[j] + hi[j]);
      const R step = m[j] - mn;
      m[j] = mn;
      if (r_abs(step) <= tau * s) {
        act[j] = false;
        vx[j] = gs[j] * m[j];
      }
      any |= act[j];
    }
  }
#pragma unroll
  for (int j = 0; j < N; ++j)
    if (act[j]) vx[j] = gs[j] * m[j];  // the iteration cap (the bracket holds the root)
}

// Direction with cos(theta) = 1 - 2 ua about x and azimuth 2 pi ub.
template <typename R>
__device__ __forceinline__ void isotropic(R speed, R ua, R ub, R two_pi, R& vx, R& vy, R& vz) {
  const R ct = (R)1 - (R)2 * ua;
  const R st = r_sqrt(r_max((R)0, ((R)1 - ct) * ((R)1 + ct)));
  const R ph = two_pi * ub;
  vx = speed * ct;
  vy = speed * (st * r_cos(ph));
  vz = speed * (st * r_sin(ph));
}

// Turn the unit vector u by polar angle chi (cos cc, sin sc) and azimuth
// (cos cp, sin sp) about itself; perpendicular frame from the x axis, or the
// z axis when |ux| > 0.99.
template <typename R>
__device__ __forceinline__ void rotate(R& ux, R& uy, R& uz, R cc, R sc, R cp, R sp) {
  R nx, ny, nz;
  if (r_abs(ux) <= (R)0.99) {
    const R w = r_sqrt(((R)1 - ux) * ((R)1 + ux));
    nx = ux * cc + sc * (cp * w);
    ny = uy * cc + sc * ((uz * sp - ux * (uy * cp)) / w);
    nz = uz * cc - sc * ((uy * sp + ux * (uz * cp)) / w);
  } else {
    const R w = r_sqrt(((R)1 - uz) * ((R)1 + uz));
    nx = ux * cc + sc * ((uy * sp - uz * (ux * cp)) / w);
    ny = uy * cc - sc * ((ux * sp + uz * (uy * cp)) / w);
    nz = uz * cc + sc * (cp * w);
  }
  ux = nx;
  uy = ny;
  uz = nz;
}

// Fixed-point charge of a marker: round(w 2^shift) to the nearest integer,
// ties to even (the value llrint gives), for wscale = 2^shift: w * 2^shift is
// exact in either type (a power-of-two scaling that stays in range) and the
// conversion rounds it once.
__device__ __forceinline__ long long fixed_charge(float w, float wscale) {
  return __float2ll_rn(w * wscale);
}
__device__ __forceinline__ long long fixed_charge(double w, double wscale) {
  return __double2ll_rn(w * wscale);
}

// Split a fixed-point charge between the two nodes of the marker's cell with
// 24-bit linear weights: the right node gets floor(Q f / 2^24),
// f = trunc(offset 2^24).
__device__ __forceinline__ long long right_share(long long Q, float off) {
  const long long f = (long long)__float2int_rz(off * 16777216.0f);
  return (Q * f) >> 24;
}
__device__ __forceinline__ long long right_share(long long Q, double off) {
  const long long f = (long long)__double2int_rz(off * 16777216.0);
  return (Q * f) >> 24;
}

}  // namespace slpic

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, cp.async.bulk) and mbarriers, as inline PTX.
// Global and shared addresses must be 16-byte aligned and sizes multiples of
// 16 bytes.
// ---------------------------------------------------------------------------
namespace slpic {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// One poll of the barrier phase; true once the phase with parity `phase` is
// complete.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void bulk_store(void* dst_gmem, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
               "r"(smem_u32(src_smem)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until every committed bulk store has finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Wait until every committed bulk store has completed.
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Order this thread's generic-proxy shared-memory accesses with later
// async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace slpic

namespace slpic {

// Polls a bounded wait makes before it gives up: the context's limit, or
// kSpinLimit.
__device__ __forceinline__ uint32_t spin_limit(const Control* ctrl) {
  const uint32_t l = *((volatile const unsigned int*)&ctrl->spin_limit);
  return l ? l : kSpinLimit;
}

// Ordered scan over chunks taken in increasing order (decoupled look-back),
// called by all 32 lanes of one warp: chunk c of a scan whose first chunk is
// `first` publishes its aggregate, then reads the records of up to 32
// predecessors at a time (lane l: chunk c - 1 - l - 32 m), adds them down to
// the nearest inclusive prefix, publishes its own inclusive prefix and returns
// its exclusive prefix.  A chunk publishes its aggregate before it waits and
// chunks go to running CTAs in order, so every wait ends; waits are bounded
// anyway and a time-out raises kErrTimeout (the result is then meaningless).
__device__ __forceinline__ void chunk_publish(ChunkStatus* t, uint32_t v, bool inclusive,
                                              unsigned int epoch) {
  if (inclusive) t->incl = v;
  else t->agg = v;
  cuda::atomic_ref<unsigned int, cuda::thread_scope_device> f(t->flag);
  f.store((epoch << 2) | (inclusive ? 2u : 1u), cuda::memory_order_release);
}

__device__ __forceinline__ uint32_t chunk_lookback(ChunkStatus* st, unsigned int c,
                                                   unsigned int first, uint32_t agg,
                                                   unsigned int epoch, Control* ctrl) {
  const int lane = threadIdx.x & 31;
  if (c == first) {
    if (lane == 0) chunk_publish(st + c, agg, true, epoch);
    return 0;
  }
  if (lane == 0) chunk_publish(st + c, agg, false, epoch);
  const uint32_t limit = spin_limit(ctrl);
  uint32_t excl = 0;
  long long top = (long long)c - 1;  // nearest predecessor not yet added
  bool timed_out = false;
  while (top >= (long long)first) {
    const long long j = top - lane;
    const bool valid = j >= (long long)first;
    unsigned int fv = 0;
    uint32_t polls = 0;
    if (valid) {
      cuda::atomic_ref<unsigned int, cuda::thread_scope_device> f(st[j].flag);
      fv = f.load(cuda::memory_order_acquire);
      while ((fv >> 2) != epoch || (fv & 3u) == 0u) {
        if (++polls > limit || *((volatile int*)&ctrl->error) == kErrTimeout) {
          timed_out = true;
          break;
        }
        __nanosleep(32);
        fv = f.load(cuda::memory_order_acquire);
      }
    }
    if (__any_sync(0xFFFFFFFFu, timed_out)) {
      if (lane == 0) atomicCAS(&ctrl->error, 0, kErrTimeout);
      timed_out = true;
      break;
    }
    const uint32_t maxp = __reduce_max_sync(0xFFFFFFFFu, polls);
    if (lane == 0 && maxp) {
      atomicAdd(&ctrl->spin_waits, 1u);
      atomicMax(&ctrl->spin_max, maxp);
    }
    const bool incl = valid && (fv & 3u) == 2u;
    uint32_t v = 0;
    if (valid) v = incl ? *((volatile unsigned int*)&st[j].incl)
                        : *((volatile unsigned int*)&st[j].agg);
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, incl);
    // lanes up to the nearest inclusive record (or the whole window)
    const int stop = b ? __ffs(b) - 1 : 31;
    if (lane > stop) v = 0;
    excl += __reduce_add_sync(0xFFFFFFFFu, v);
    if (b) break;
    top -= 32;
  }
  if (lane == 0) chunk_publish(st + c, excl + agg, true, epoch);
  return excl;
}

}  // namespace slpic
