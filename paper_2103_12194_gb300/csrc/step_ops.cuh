// Pieces of one SLPIC-MCC step shared by the batched kernels (push.cu,
// collide.cu, finish.cu) and the single-CTA path (small.cu): the
// electrode and emission handling of a marker, the collision of a
// candidate and the births it makes, block scans, the exact integer sums
// of the Poisson solve and the commit of a step's tallies.  Both paths call
// the same functions, so a marker takes the same arithmetic in each.
#pragma once

#include "device_common.cuh"
#include "slpic_internal.h"

namespace slpic {

namespace {

// A marker left the gap: tally the flux through the electrode (Eq. j); an ion
// at the cathode emits an electron with probability gamma.  Returns true when
// an electron is emitted.  Rare; kept out of line.
template <typename R>
__device__ __noinline__ bool absorb(const InstDev& P, int sp, int side, R wj, uint32_t id,
                                    uint32_t step, unsigned long long* acc, R vx, R vy, R vz) {
  const StepConsts<R>& K = consts<R>(P);
  const long long Qw = fixed_charge(wj, K.wscale);
  atomicAdd(&acc[ACC_NABS + sp * 2 + side], 1ull);
  atomicAdd(&acc[ACC_WABS + sp * 2 + side], (unsigned long long)Qw);
  if (sp != kIon || side != 0) return false;
  atomicAdd(&acc[ACC_WCATH], (unsigned long long)Qw);
  // secondary-electron yield: constant, or Eq. sey at the ion's kinetic
  // energy (exponent 0.05 below 700 eV, 0.72 from 700 eV on)
  R g = K.gamma;
  if (P.emission_model == 1) {
    const R eps_i = (vx * vx + vy * vy + vz * vz) * K.K_Ei;
    const R expo = eps_i < (R)700 ? (R)0.05 : (R)0.72;
    g = (R)0.09 * r_pow(eps_i / (R)700, expo);
  }
  if (!(id & kGenBit)) {
    atomicAdd(&acc[ACC_WCATH0], (unsigned long long)Qw);
    atomicAdd(&acc[ACC_GWCATH0], (unsigned long long)fixed_charge(g * wj, K.wscale));
  }
  const uint4 rr =
      philox4x32_10(make_uint4(id, step, P.ctr_inst * 2u + 1u, 0u), P.key0, P.key1);
  if (!P.emit || !(uniform01r<R>(rr.x) < g)) return false;
  atomicAdd(&acc[ACC_SEE], 1ull);
  atomicAdd(&acc[ACC_WSEE], (unsigned long long)Qw);
  return true;
}

// Stage an electron emitted at the cathode (x = 0, at rest, the ion's w_j);
// with kDeposit, deposit it too.
template <typename R, bool kDeposit = true>
__device__ __noinline__ void stage_emission(const InstDev& P, size_t o, R wj) {
  const SoAT<R> sb = soa_as<R>(P.sp[kElectron].stage_b);
  sb.cell[o] = 0;
  sb.off[o] = (R)0;
  sb.vx[o] = (R)0;
  sb.vy[o] = (R)0;
  sb.vz[o] = (R)0;
  sb.wj[o] = wj;
  sb.id[o] = kGenBit;
  // at rest: beta = 1, all the charge on node 0
  if (kDeposit)
    atomicAdd(P.rho_acc[kElectron], (unsigned long long)fixed_charge(wj, consts<R>(P).wscale));
}

// Interpolated cumulative cross sections at eps (linear between the nodes of
// the octave-uniform grid, held constant outside it): xs[0 .. n_exc + 1].
// The node index and the fraction come exactly from the exponent and
// mantissa bits of eps.
__device__ __forceinline__ void xsec(const InstDev& P, float eps, float* xs) {
  const StepConsts<float>& K = P.c32;
  int j;
  float t;
  if (!(eps >= K.e_lo)) {
    j = 0;
    t = 0.0f;
  } else if (eps >= K.e_hi) {
    j = P.tab_nodes - 1;
    t = 0.0f;
  } else {
    const uint32_t b = __float_as_uint(eps);
    const int octave = (int)(b >> 23) - 127 - P.tab_lo_exp2;
    const uint32_t mant = b & 0x7FFFFFu;
    const int sh = 23 - P.tab_log2_sub;
    j = (octave << P.tab_log2_sub) + (int)(mant >> sh);
    const float scale = __int_as_float((127 - sh) << 23);  // 2^-sh
    t = __uint2float_rn(mant & ((1u << sh) - 1u)) * scale;
  }
  const int st = P.tab_stride;
  const float4 a = __ldg(P.table + j * st);
  const float4 c = __ldg(P.table + (j + 1) * st);
  xs[0] = a.x + t * (c.x - a.x);
  xs[1] = a.y + t * (c.y - a.y);
  xs[2] = a.z + t * (c.z - a.z);
  xs[3] = a.w + t * (c.w - a.w);
  if (st > 1) {
    const float4 a1 = __ldg(P.table + j * st + 1);
    const float4 c1 = __ldg(P.table + (j + 1) * st + 1);
    xs[4] = a1.x + t * (c1.x - a1.x);
  }
}

__device__ __forceinline__ void xsec(const InstDev& P, double eps, double* xs) {
  const StepConsts<double>& K = P.c64;
  int j;
  double t;
  if (!(eps >= K.e_lo)) {
    j = 0;
    t = 0.0;
  } else if (eps >= K.e_hi) {
    j = P.tab_nodes - 1;
    t = 0.0;
  } else {
    const unsigned long long b = (unsigned long long)__double_as_longlong(eps);
    const int octave = (int)(b >> 52) - 1023 - P.tab_lo_exp2;
    const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
    const int sh = 52 - P.tab_log2_sub;
    j = (octave << P.tab_log2_sub) + (int)(mant >> sh);
    const double scale = __longlong_as_double((long long)(1023 - sh) << 52);  // 2^-sh
    t = (double)(mant & ((1ull << sh) - 1ull)) * scale;
  }
  const TabNode64& a = P.table64[j];
  const TabNode64& c = P.table64[j + 1];
  const int n_proc = P.n_exc + 2;
#pragma unroll
  for (int k = 0; k < kMaxProc; ++k)
    if (k < n_proc) xs[k] = a.s[k] + t * (c.s[k] - a.s[k]);
}

template <typename R>
__device__ __forceinline__ void deposit(unsigned long long* rho, int cell, R off, long long Q) {
  const long long right = right_share(Q, off);
  const long long left = Q - right;
  if (left) atomicAdd(rho + cell, (unsigned long long)left);
  if (right) atomicAdd(rho + cell + 1, (unsigned long long)right);
}

template <typename R>
struct Velocity {
  R vx, vy, vz;
};

// Process of a null-collision candidate (speed v1, v1^2 = s1): u = the four
// uniforms of its Philox4x32 block rr (u[0] is unused: the candidate test drew
// from Philox2x32); u[1] P0 is compared with the cumulative rates
// n_g sigma_k(eps) beta v dt.  Returns 0 elastic, 1 excitation, 2 ionization,
// 3 null, with eps the candidate's energy and k its index in the cumulative
// list (excitation level k for proc 1).
template <typename R>
__device__ __forceinline__ int choose_process(const InstDev& P, R vlim, R v1, R s1, uint4 rr,
                                              unsigned long long* acc, R (&u)[4], R& eps,
                                              int& k_out) {
  const StepConsts<R>& K = consts<R>(P);
  uniform4<R>(rr, u);
  R vb = v1 > vlim ? vlim : v1;
  if (vb > K.vb_cap) {
    vb = K.vb_cap;
    atomicAdd(&acc[ACC_MAJ], 1ull);
  }
  const R c = K.ndt * vb;
  eps = s1 * K.K_E;
  R xs[kMaxProc];
  xsec(P, eps, xs);
  const R rsel = u[1] * K.P0;
  // the first process whose cumulative rate exceeds the draw: elastic,
  // excitation level 1..n_exc, ionization; none: a null collision
  const int n_proc = P.n_exc + 2;
  int k = 0;
  while (k < n_proc && !(rsel < c * xs[k])) ++k;
  k_out = k;
  return k == n_proc ? 3 : (k == 0 ? 0 : (k <= P.n_exc ? 1 : 2));
}

// Elastic scattering of an electron of velocity v (speed v1, energy eps) by
// the Vahedi-Surendra angles (u2: polar, u3: azimuth) with the recoil loss.
template <typename R>
__device__ __forceinline__ Velocity<R> scatter_elastic(const StepConsts<R>& K, R kv, R vx, R vy,
                                                       R vz, R v1, R eps, R u2, R u3) {
  // Vahedi-Surendra: cos chi = (2 + eps - 2 (1 + eps)^u) / eps, with
  // 1 - cos chi and 1 + cos chi each formed without cancellation so that
  // sin chi keeps its relative precision at both ends
  const R L = r_log1p(eps);
  const R em = r_expm1(u2 * L);
  const R ep = -r_expm1(-((R)1 - u2) * L);
  R omc = (em + em) / eps;
  R opc = (((R)1 + eps) * (ep + ep)) / eps;
  omc = r_min((R)2, r_max((R)0, omc));
  opc = r_min((R)2, r_max((R)0, opc));
  const R cc = omc <= (R)1 ? (R)1 - omc : opc - (R)1;
  const R sc = r_sqrt(omc * opc);
  const R ph = K.two_pi * u3;
  const R cp = r_cos(ph), sn = r_sin(ph);
  const R e_new = eps * ((R)1 - K.R2 * omc);
  R ux = vx / v1, uy = vy / v1, uz = vz / v1;
  rotate(ux, uy, uz, cc, sc, cp, sn);
  const R vn = r_sqrt(e_new * kv);
  return {vn * ux, vn * uy, vn * uz};
}

// Excitation of level k: the threshold removed, an isotropic direction.
template <typename R>
__device__ __forceinline__ Velocity<R> scatter_excitation(const StepConsts<R>& K, R kv, R eps, int k,
                                                          R u2, R u3, unsigned long long* acc) {
  R e_new = eps - K.e_ex[k - 1];
  if (e_new < (R)0) {
    e_new = (R)0;
    atomicAdd(&acc[ACC_CLAMP], 1ull);
  }
  Velocity<R> o;
  isotropic(r_sqrt(e_new * kv), u2, u3, K.two_pi, o.vx, o.vy, o.vz);
  return o;
}

// Ionization: the excess energy shared between the primary (isotropic) and
// the secondary (*es_out, block 1 of the primary's draws), the flux weight
// of the pair tallied.
template <typename R>
__device__ __forceinline__ Velocity<R> scatter_ionization(const InstDev& P, R kv, R eps, R u2,
                                                          R u3, uint32_t id, uint32_t step, R wj,
                                                          unsigned long long* acc, R* es_out) {
  const StepConsts<R>& K = consts<R>(P);
  R e_av = eps - K.e_io;
  if (e_av < (R)0) {
    e_av = (R)0;
    atomicAdd(&acc[ACC_CLAMP], 1ull);
  }
  atomicAdd(&acc[ACC_WIONZ], (unsigned long long)fixed_charge(wj, K.wscale));
  const uint4 r1 =
      philox4x32_10(make_uint4(id, step, P.ctr_inst * 2u, 1u), P.key0, P.key1);
  const R es = uniform01r<R>(r1.x) * e_av;
  const R ep = e_av - es;
  Velocity<R> o;
  isotropic(r_sqrt(ep * kv), u2, u3, K.two_pi, o.vx, o.vy, o.vz);
  *es_out = es;
  return o;
}

// Choose the process and scatter (Sec. III and IV).  Returns the new
// velocity; *proc_out = 0 elastic, 1 excitation, 2 ionization, 3 null
// (velocity unchanged).  The caller counts the candidate and its process
// (ACC_CAND, ACC_COLL0 + proc for proc < 3).  Kept out of line: the
// single-CTA path calls it from several unrolled rows, and one copy of the
// long scattering code keeps that latency-bound kernel's instruction
// footprint small.
template <typename R>
__device__ __noinline__ Velocity<R> collide(const InstDev& P, R kv, R vlim, R vx, R vy, R vz, R v1, R s1,
                               uint4 rr, uint32_t id, uint32_t step, R wj,
                               unsigned long long* acc, R* e_sec_out, int* proc_out) {
  R u[4], eps;
  int k;
  const int proc = choose_process<R>(P, vlim, v1, s1, rr, acc, u, eps, k);
  *proc_out = proc;
  if (proc == 0) return scatter_elastic<R>(consts<R>(P), kv, vx, vy, vz, v1, eps, u[2], u[3]);
  if (proc == 1) return scatter_excitation<R>(consts<R>(P), kv, eps, k, u[2], u[3], acc);
  if (proc == 2) return scatter_ionization<R>(P, kv, eps, u[2], u[3], id, step, wj, acc, e_sec_out);
  return {vx, vy, vz};
}

// Write the electron and Ar+ born by an ionization at slots pe (electron
// store) and pi (ion store) with their serial numbers, and (kDeposit) deposit
// both.  The secondary gets energy es along an isotropic direction (block 1
// of the primary's draws); the ion a gas-temperature Maxwellian (Box-Muller
// on block 2).
template <typename R, bool kDeposit = true>
__device__ void born_pair(const InstDev& P, const SoAT<R>& me, const SoAT<R>& mi, uint32_t pe,
                          uint32_t pi, int cell, R off, R wj, uint32_t id, uint32_t step, R es,
                          uint32_t serial_e, uint32_t serial_i) {
  const StepConsts<R>& K = consts<R>(P);
  const uint32_t gen = id & kGenBit;
  const uint4 r1 = philox4x32_10(make_uint4(id, step, P.ctr_inst * 2u, 1u), P.key0, P.key1);
  R bx, by, bz;
  isotropic(r_sqrt(es * K.K_V[kElectron]), uniform01r<R>(r1.y), uniform01r<R>(r1.z), K.two_pi,
            bx, by, bz);
  me.cell[pe] = cell;
  me.off[pe] = off;
  me.vx[pe] = bx;
  me.vy[pe] = by;
  me.vz[pe] = bz;
  me.wj[pe] = wj;
  me.id[pe] = gen | (serial_e & kSerialMask);
  if (kDeposit)
    deposit(P.rho_acc[kElectron], cell, off,
            fixed_charge(beta_of(r_sqrt(bx * bx + by * by + bz * bz), K.vlim[kElectron]) * wj,
                         K.wscale));
  const uint4 r2 = philox4x32_10(make_uint4(id, step, P.ctr_inst * 2u, 2u), P.key0, P.key1);
  R g[4];
  uniform4<R>(r2, g);
  const R rr1 = r_sqrt((R)-2 * r_log(g[0]));
  const R rr2 = r_sqrt((R)-2 * r_log(g[2]));
  const R a1 = K.two_pi * g[1], a2 = K.two_pi * g[3];
  const R ix = K.sigT_ion * (rr1 * r_cos(a1));
  const R iy = K.sigT_ion * (rr1 * r_sin(a1));
  const R iz = K.sigT_ion * (rr2 * r_cos(a2));
  mi.cell[pi] = cell;
  mi.off[pi] = off;
  mi.vx[pi] = ix;
  mi.vy[pi] = iy;
  mi.vz[pi] = iz;
  mi.wj[pi] = wj;
  mi.id[pi] = gen | (serial_i & kSerialMask);
  if (kDeposit)
    deposit(P.rho_acc[kIon], cell, off,
            fixed_charge(beta_of(r_sqrt(ix * ix + iy * iy + iz * iz), K.vlim[kIon]) * wj,
                         K.wscale));
}

// Slot after the last live marker of a store (the particle kernel has
// compacted every tile of this step).
__device__ __forceinline__ uint32_t tail_slot(const SpeciesDev& S, const SpeciesState& st) {
  return st.n_tiles ? (st.n_tiles - 1) * (uint32_t)kTile + S.fill[st.cur][st.n_tiles - 1]
                    : 0u;
}

template <typename R>
__device__ __forceinline__ void write_marker(const SoAT<R>& d, size_t o, int cell, R off, R vx,
                                             R vy, R vz, R wj, uint32_t id) {
  d.cell[o] = cell;
  d.off[o] = off;
  d.vx[o] = vx;
  d.vy[o] = vy;
  d.vz[o] = vz;
  d.wj[o] = wj;
  d.id[o] = id;
}

// Record of null-collision candidate i of an electron store (the tile's
// queue slot tbase + rank): in float two 16-byte stores of one sector.
__device__ __forceinline__ void put_cand(void* crec, size_t i, int cell, float off, float vx,
                                         float vy, float vz, float wj, uint32_t id,
                                         uint32_t slot) {
  float4* p = reinterpret_cast<float4*>(reinterpret_cast<CandRec<float>*>(crec) + i);
  p[0] = make_float4(__int_as_float(cell), off, vx, vy);
  p[1] = make_float4(vz, wj, __uint_as_float(id), __uint_as_float(slot));
}
__device__ __forceinline__ void put_cand(void* crec, size_t i, int cell, double off, double vx,
                                         double vy, double vz, double wj, uint32_t id,
                                         uint32_t slot) {
  CandRec<double> c;
  c.cell = cell;
  c.id = id;
  c.off = off;
  c.vx = vx;
  c.vy = vy;
  c.vz = vz;
  c.wj = wj;
  c.slot = slot;
  c.pad = 0u;
  reinterpret_cast<CandRec<double>*>(crec)[i] = c;
}

template <typename R>
__device__ __forceinline__ CandRec<R> get_cand(const void* crec, size_t i) {
  return reinterpret_cast<const CandRec<R>*>(crec)[i];
}

constexpr int kFinThreads = 1024;

__device__ __forceinline__ long long shfl_up(long long v, int o) {
  return __shfl_up_sync(0xFFFFFFFFu, v, o);
}
__device__ __forceinline__ __int128 shfl_up(__int128 v, int o) {
  const unsigned long long lo = __shfl_up_sync(0xFFFFFFFFu, (unsigned long long)v, o);
  const long long hi = __shfl_up_sync(0xFFFFFFFFu, (long long)(v >> 64), o);
  return (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | lo);
}

// Inclusive block scan over a CTA of kThreads threads: shuffle scans within
// the warps, then one warp scans the warp totals (buf holds 32 entries).
// Integer sums, so exact.
template <typename T, int kThreads = kFinThreads>
__device__ T block_incl_scan(T v, T* buf) {
  static_assert(kThreads % 32 == 0 && kThreads <= 1024, "whole warps, at most 32");
  constexpr int kWarps = kThreads / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    const T y = shfl_up(v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) buf[w] = v;
  __syncthreads();
  if (w == 0) {
    T t = lane < kWarps ? buf[lane] : T(0);
    for (int o = 1; o < 32; o <<= 1) {
      const T y = shfl_up(t, o);
      if (lane >= o) t += y;
    }
    if (lane < kWarps) buf[lane] = t;
  }
  __syncthreads();
  const T r = v + (w ? buf[w - 1] : T(0));
  __syncthreads();
  return r;
}

// Net deposit (ions minus electrons) at node k of the last step: from the
// CTA's shared copy when there is one, else from the last deposit.
__device__ __forceinline__ long long net_at(const InstDev& P, const long long* s_net, int k) {
  return s_net ? s_net[k] : P.rho_last[kIon][k] - P.rho_last[kElectron][k];
}

// The exact integer sums of the 1D Poisson solve over the last step's net
// deposit (all threads of a kThreads CTA; thread t covers k = k0 ..
// k0 + chunk - 1 of 1..N): returns D_1 = (V + C J_N) / N and writes I_{k0}.
template <int kThreads = kFinThreads>
__device__ double poisson_d1(const InstDev& P, const long long* s_net, int k0, int chunk,
                             long long* s_i64, __int128* s_i128, long long* I_k0) {
  const int N = P.n_cells;
  long long loc = 0;
  for (int k = k0; k < k0 + chunk && k <= N - 1; ++k) loc += net_at(P, s_net, k);
  const long long inc = block_incl_scan<long long, kThreads>(loc, s_i64);
  long long Ik = inc - loc;  // I_k at the chunk start (exclusive of net_k)
  *I_k0 = Ik;
  __int128 locJ = 0;
  for (int k = k0; k < k0 + chunk && k <= N; ++k) {
    locJ += (__int128)Ik;
    if (k <= N - 1) Ik += net_at(P, s_net, k);
  }
  const __int128 incJ = block_incl_scan<__int128, kThreads>(locJ, s_i128);
  // one thread forms D_1 (FP64 is scarce on this part) and shares it
  __shared__ double s_D1;
  if (threadIdx.x == kThreads - 1) s_D1 = (P.V + P.pois_C * (double)incJ) / (double)N;
  __syncthreads();
  const double D1 = s_D1;
  __syncthreads();
  return D1;
}

// The node field of instance P's last Poisson solve from its exact integer
// sums (k_finish leaves I_k and D_1): the centred difference of phi,
// E_k = -(2 D_1 - C (I_k + I_{k+1})) / (2 dx), one-sided at the electrodes,
// for the nodes k = k0, k0 + stride, ...
__device__ __forceinline__ void poisson_field(const InstDev& P, int k0, int stride) {
  const int N = P.n_cells;
  const double D1 = *P.pois_D1;
  const double C = P.pois_C;
  const double inv2dx = 1.0 / (2.0 * P.dx);
  const double twoD1 = D1 + D1;
  for (int k = k0; k <= N; k += stride) {
    double e;
    if (k == 0) {
      e = -D1 / P.dx;  // I_1 = 0: D_1
    } else if (k <= N - 1) {
      e = -(twoD1 - C * (double)(P.pois_I[k] + P.pois_I[k + 1])) * inv2dx;
    } else {
      e = -(D1 - C * (double)P.pois_I[k]) / P.dx;  // k = N
    }
    P.E64[k] = e;
    P.E32[k] = (float)e;
  }
}

// Record of one step (TallyRec) from its accumulators q: thread t < kTallySlots
// writes 8-byte slot t to the history ring and the totals.  Slot layout: 0
// step, 1-2 n_live, 3-4 w_live, 5-7 n_coll, 8 n_candidates, 9-12 n_abs, 13-16
// w_abs, 17 n_see, 18 w_see, 19 w_ionz, 20 w_cath_ion, 21 w_cath_ion_gen0, 22
// n_clamp, 23 n_majorant, 24 marker_steps, 25 w_gain_gen0; slots 0-4 are
// states (replaced in the totals), the others sums.  n_live_* are the counts
// after the step; w_live (fixed point, per species) is updated by its changes,
// and ion_steps gains the step's live ions.
constexpr int kTallySlots = (int)(sizeof(TallyRec) / 8);
static_assert(kTallySlots == 26, "TallyRec layout");

__device__ __forceinline__ void commit_tally_slot(const InstDev& P, int t,
                                                  const unsigned long long* q, uint32_t step,
                                                  long long n_steps_done, uint32_t n_live_e,
                                                  uint32_t n_live_i, unsigned long long* w_live,
                                                  long long* ion_steps) {
  const double unit = 1.0 / P.c64.wscale;
  long long iv = 0;
  double dv = 0.0;
  bool is_double = false;
  if (t == 0) {
    iv = step;
  } else if (t <= 2) {
    iv = t == 1 ? n_live_e : n_live_i;
    if (t == 2) *ion_steps += iv;
  } else if (t <= 4) {
    // live weight by its changes: minus what left through the electrodes,
    // plus the births (ionization pairs; emitted electrons)
    const int sp = t - 3;
    unsigned long long w = w_live[sp] - q[ACC_WABS + 2 * sp] - q[ACC_WABS + 2 * sp + 1] +
                           q[ACC_WIONZ] + (sp == 0 ? q[ACC_WSEE] : 0ull);
    w_live[sp] = w;
    dv = (double)(long long)w * unit;
    is_double = true;
  } else if (t <= 7) {
    iv = (long long)q[ACC_COLL0 + t - 5];
  } else if (t == 8) {
    iv = (long long)q[ACC_CAND];
  } else if (t <= 12) {
    iv = (long long)q[ACC_NABS + t - 9];
  } else if (t <= 16) {
    dv = (double)(long long)q[ACC_WABS + t - 13] * unit;
    is_double = true;
  } else if (t == 17) {
    iv = (long long)q[ACC_SEE];
  } else if (t <= 21) {
    const int acc_of[4] = {ACC_WSEE, ACC_WIONZ, ACC_WCATH, ACC_WCATH0};
    dv = (double)(long long)q[acc_of[t - 18]] * unit;
    is_double = true;
  } else if (t == 22) {
    iv = (long long)q[ACC_CLAMP];
  } else if (t == 23) {
    iv = (long long)q[ACC_MAJ];
  } else if (t == 24) {
    iv = (long long)q[ACC_MSTEPS];
  } else {
    dv = (double)(long long)q[ACC_GWCATH0] * unit;
    is_double = true;
  }
  long long* ring = reinterpret_cast<long long*>(P.ring + n_steps_done % P.ring_len);
  long long* tot = reinterpret_cast<long long*>(P.total);
  if (is_double) {
    reinterpret_cast<double*>(ring)[t] = dv;
    if (t <= 4) reinterpret_cast<double*>(tot)[t] = dv;
    else reinterpret_cast<double*>(tot)[t] += dv;
  } else {
    ring[t] = iv;
    if (t <= 4) tot[t] = iv;
    else tot[t] += iv;
  }
}

}  // namespace

}  // namespace slpic
