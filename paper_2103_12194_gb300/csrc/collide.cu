// Monte-Carlo collisions of the null-collision candidates queued by the
// particle kernel (Sec. III and IV): for a candidate (an electron that drew
// u < P0 this step) the process is chosen by comparing u' P0 with the
// cumulative rates n_g sigma_k(eps) beta v dt (Eq. SLPICcollisionNumber with
// beta_n = 1, whole-marker collisions); elastic collisions scatter by the
// Vahedi-Surendra angles with the recoil loss, excitation removes its
// threshold and scatters isotropically, ionization shares the excess energy
// and stages the born electron and Ar+ (same position, same flux weight).
// Each candidate is then deposited with its new density weight.
//
// One warp per tile, one lane per candidate: the scattering path is long and
// latency-bound, and running it here, over every candidate of the step at
// once, keeps it away from the streaming particle kernel.  Births are ranked
// in slot order inside their tile with ballots, so their order (and the
// serial numbers they get when appended) does not depend on scheduling.
#include "device_common.cuh"
#include "slpic_internal.h"

namespace slpic {

namespace {

constexpr int kCollThreads = 256;

// Interpolated cumulative cross sections at eps (linear between the nodes of
// the octave-uniform grid, held constant outside it).
__device__ __forceinline__ void xsec(const InstDev& P, float eps, float& s1, float& s2,
                                     float& s3) {
  int j;
  float t;
  if (!(eps >= P.e_lo)) {
    j = 0;
    t = 0.0f;
  } else if (eps >= P.e_hi) {
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
  const float4 a = __ldg(P.table + j);
  const float4 c = __ldg(P.table + j + 1);
  s1 = a.x + t * (c.x - a.x);
  s2 = a.y + t * (c.y - a.y);
  s3 = a.z + t * (c.z - a.z);
}

__device__ __forceinline__ void deposit(unsigned long long* rho, int cell, float off,
                                        long long Q) {
  const long long right = right_share(Q, off);
  const long long left = Q - right;
  if (left) atomicAdd(rho + cell, (unsigned long long)left);
  if (right) atomicAdd(rho + cell + 1, (unsigned long long)right);
}

struct Velocity {
  float vx, vy, vz;
};

// Choose the process with u[1] against the cumulative rates and scatter.
// Returns the new velocity; *proc_out = 0 elastic, 1 excitation,
// 2 ionization, 3 null (velocity unchanged).
__device__ Velocity collide(const InstDev& P, float kv, float vlim, float vx, float vy,
                            float vz, float v1, float s1, uint4 rr, uint32_t id, uint32_t step,
                            float wj, unsigned long long* acc, float* e_sec_out,
                            int* proc_out) {
  float u[4];
  uniform4(rr, u);
  atomicAdd(&acc[ACC_CAND], 1ull);
  float vb = v1 > vlim ? vlim : v1;
  if (vb > P.vb_cap) {
    vb = P.vb_cap;
    atomicAdd(&acc[ACC_MAJ], 1ull);
  }
  const float c = P.ndt * vb;
  const float eps = s1 * P.K_E;
  float x1, x2, x3;
  xsec(P, eps, x1, x2, x3);
  const float rsel = u[1] * P.P0;
  int proc = 3;
  if (rsel < c * x1) proc = 0;
  else if (rsel < c * x2) proc = 1;
  else if (rsel < c * x3) proc = 2;
  *proc_out = proc;
  Velocity o = {vx, vy, vz};
  if (proc == 3) return o;
  atomicAdd(&acc[ACC_COLL0 + proc], 1ull);
  if (proc == 0) {
    // Vahedi-Surendra: cos chi = (2 + eps - 2 (1 + eps)^u) / eps, with
    // 1 - cos chi and 1 + cos chi each formed without cancellation so that
    // sin chi keeps its relative precision at both ends
    const float L = log1pf(eps);
    const float em = expm1f(u[2] * L);
    const float ep = -expm1f(-(1.0f - u[2]) * L);
    float omc = (em + em) / eps;
    float opc = ((1.0f + eps) * (ep + ep)) / eps;
    omc = fminf(2.0f, fmaxf(0.0f, omc));
    opc = fminf(2.0f, fmaxf(0.0f, opc));
    const float cc = omc <= 1.0f ? 1.0f - omc : opc - 1.0f;
    const float sc = sqrtf(omc * opc);
    const float ph = P.two_pi * u[3];
    const float cp = cosf(ph), sn = sinf(ph);
    const float e_new = eps * (1.0f - P.R2 * omc);
    float ux = vx / v1, uy = vy / v1, uz = vz / v1;
    rotate(ux, uy, uz, cc, sc, cp, sn);
    const float vn = sqrtf(e_new * kv);
    o.vx = vn * ux;
    o.vy = vn * uy;
    o.vz = vn * uz;
  } else if (proc == 1) {
    float e_new = eps - P.e_ex;
    if (e_new < 0.0f) {
      e_new = 0.0f;
      atomicAdd(&acc[ACC_CLAMP], 1ull);
    }
    isotropic(sqrtf(e_new * kv), u[2], u[3], P.two_pi, o.vx, o.vy, o.vz);
  } else {
    float e_av = eps - P.e_io;
    if (e_av < 0.0f) {
      e_av = 0.0f;
      atomicAdd(&acc[ACC_CLAMP], 1ull);
    }
    atomicAdd(&acc[ACC_WIONZ], (unsigned long long)fixed_charge(wj, P.charge_shift));
    const uint4 r1 =
        philox4x32_10(make_uint4(id, step, P.ctr_inst * 2u, 1u), P.key0, P.key1);
    const float es = uniform01(r1.x) * e_av;
    const float ep = e_av - es;
    isotropic(sqrtf(ep * kv), u[2], u[3], P.two_pi, o.vx, o.vy, o.vz);
    *e_sec_out = es;
  }
  return o;
}

// Stage the electron and ion born by an ionization in slot o of the staging
// stores, and deposit both.
__device__ void stage_ionization(const InstDev& P, size_t o, int cell, float off, float wj,
                                 uint32_t id, uint32_t step, float es) {
  const SpeciesDev& SE = P.sp[kElectron];
  const SpeciesDev& SI = P.sp[kIon];
  const uint32_t gen = id & kGenBit;
  const uint4 r1 = philox4x32_10(make_uint4(id, step, P.ctr_inst * 2u, 1u), P.key0, P.key1);
  float bx, by, bz;
  isotropic(sqrtf(es * SE.K_V), uniform01(r1.y), uniform01(r1.z), P.two_pi, bx, by, bz);
  SE.stage_a.cell[o] = cell;
  SE.stage_a.off[o] = off;
  SE.stage_a.vx[o] = bx;
  SE.stage_a.vy[o] = by;
  SE.stage_a.vz[o] = bz;
  SE.stage_a.wj[o] = wj;
  SE.stage_a.id[o] = gen;  // serial assigned when appended
  deposit(P.rho_acc[kElectron], cell, off,
          fixed_charge(beta_of(sqrtf(bx * bx + by * by + bz * bz), SE.vlim) * wj,
                       P.charge_shift));
  // born ion: gas-temperature Maxwellian (Box-Muller on block 2)
  const uint4 r2 = philox4x32_10(make_uint4(id, step, P.ctr_inst * 2u, 2u), P.key0, P.key1);
  float g[4];
  uniform4(r2, g);
  const float rr1 = sqrtf(-2.0f * logf(g[0]));
  const float rr2 = sqrtf(-2.0f * logf(g[2]));
  const float a1 = P.two_pi * g[1], a2 = P.two_pi * g[3];
  const float ix = P.sigT_ion * (rr1 * cosf(a1));
  const float iy = P.sigT_ion * (rr1 * sinf(a1));
  const float iz = P.sigT_ion * (rr2 * cosf(a2));
  SI.stage_a.cell[o] = cell;
  SI.stage_a.off[o] = off;
  SI.stage_a.vx[o] = ix;
  SI.stage_a.vy[o] = iy;
  SI.stage_a.vz[o] = iz;
  SI.stage_a.wj[o] = wj;
  SI.stage_a.id[o] = gen;
  deposit(P.rho_acc[kIon], cell, off,
          fixed_charge(beta_of(sqrtf(ix * ix + iy * iy + iz * iz), SI.vlim) * wj,
                       P.charge_shift));
}

}  // namespace

__global__ void __launch_bounds__(kCollThreads) k_collide(DeviceRefs r) {
  __shared__ unsigned long long s_acc[ACC_COUNT];
  if (*((volatile int*)&r.ctrl->error)) return;
  const int lane = threadIdx.x & 31;
  const uint32_t lanemask_lt = (1u << lane) - 1u;
  const int warps_per_cta = kCollThreads / 32;
  const unsigned int wid = blockIdx.x * warps_per_cta + (threadIdx.x >> 5);
  const unsigned int n_warps = gridDim.x * warps_per_cta;
  for (int inst = 0; inst < r.n_inst; ++inst) {
    const InstDev& P = r.inst[inst];
    const SpeciesDev& S = P.sp[kElectron];
    const SpeciesState& st = r.sstate[inst * 2 + kElectron];
    const uint32_t nt = st.n_tiles;
    const SoA m = S.buf[st.cur];
    const uint32_t step = r.istate[inst].step;
    const float kv = S.K_V, vlim = S.vlim;
    if (threadIdx.x < ACC_COUNT) s_acc[threadIdx.x] = 0ull;
    __syncthreads();
    for (uint32_t k = wid; k < nt; k += n_warps) {
      const uint32_t nc = S.n_cand[k];
      if (!nc) continue;
      const size_t base = (size_t)k * kTile;
      uint32_t ranked = 0;
      for (uint32_t c0 = 0; c0 < nc; c0 += 32) {
        const uint32_t c = c0 + lane;
        bool ionized = false;
        int cell = 0;
        float off = 0.0f, wj = 0.0f, es = 0.0f;
        uint32_t id = 0;
        if (c < nc) {
          const size_t o = base + S.cand[base + c];
          cell = m.cell[o];
          off = m.off[o];
          wj = m.wj[o];
          id = m.id[o];
          float vx = m.vx[o], vy = m.vy[o], vz = m.vz[o];
          const float s1 = vx * vx + vy * vy + vz * vz;
          const float v1 = sqrtf(s1);
          const uint4 rr =
              philox4x32_10(make_uint4(id, step, P.ctr_inst * 2u, 0u), P.key0, P.key1);
          int proc;
          const Velocity nv =
              collide(P, kv, vlim, vx, vy, vz, v1, s1, rr, id, step, wj, s_acc, &es, &proc);
          if (proc < 3) {
            vx = nv.vx;
            vy = nv.vy;
            vz = nv.vz;
            m.vx[o] = vx;
            m.vy[o] = vy;
            m.vz[o] = vz;
            ionized = proc == 2;
          }
          deposit(P.rho_acc[kElectron], cell, off,
                  fixed_charge(beta_of(sqrtf(vx * vx + vy * vy + vz * vz), vlim) * wj,
                               P.charge_shift));
        }
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, ionized);
        if (ionized)
          stage_ionization(P, base + ranked + __popc(b & lanemask_lt), cell, off, wj, id, step,
                           es);
        ranked += __popc(b);
      }
      if (lane == 0) S.births[k] = ranked;
    }
    __syncthreads();
    if (threadIdx.x < ACC_COUNT && s_acc[threadIdx.x])
      atomicAdd(P.acc + threadIdx.x, s_acc[threadIdx.x]);
    __syncthreads();
  }
}

void launch_collide(const DeviceRefs& r, int grid, cudaStream_t s) {
  k_collide<<<grid, kCollThreads, 0, s>>>(r);
}

}  // namespace slpic
