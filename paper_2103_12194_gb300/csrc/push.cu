// The particle kernel of one SLPIC-MCC step, batched over instances and
// species: gather, speed-limited kick and drift (Eqs. slpicEOMx, slpicEOMv,
// betaAbrupt), absorbing electrodes with ion-induced secondary emission
// (Sec. IV), null-collision Monte-Carlo collisions of electrons with a
// background gas (Sec. III, Eq. SLPICcollisionNumber with beta_n = 1),
// ionization births, in-place compaction of survivors, and the fixed-point
// deposit of w_p = beta w_j (Eq. Ansatz).
//
// Work decomposition.  Every (instance, species) segment is a sequence of
// tiles of kTile marker slots (tile k holds fill[k] markers).  A persistent
// grid takes tiles in increasing global order from an atomic counter; tiles
// are independent, so no CTA ever waits for another.  Per CTA the tiles go
// through a two-stage shared-memory pipeline:
//   - bulk asynchronous copies (TMA, cp.async.bulk) bring the seven SoA
//     streams of the next tile into one stage while the current tile is
//     advanced in the other;
//   - each thread advances the markers of slots t and t + kThreads in place
//     in the stage and deposits the survivors into a shared-memory copy of the
//     segment's charge grid (integer atomics); the rare collision and birth
//     work runs out of line so the common path stays small;
//   - warp ballots and one scan over the warps rank survivors and births; the
//     survivors are written back compacted and in order and stored to the
//     tile's own slots with bulk copies; births go to tile-local staging slots.
// The shared charge grid is added to global memory with integer atomics when
// the CTA moves to another segment or finishes, so the deposit is exact and
// independent of the order of the additions.
#include "device_common.cuh"
#include "slpic_internal.h"

namespace slpic {

namespace {

constexpr int kWarps = kThreads / 32;

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

struct TileInfo {
  unsigned int g;     // global tile index (>= n_tiles: none)
  int seg;            // segment = instance * 2 + species
  unsigned int k;     // tile inside the segment
  unsigned int fill;  // live markers in the tile
};

struct CtaShared {
  unsigned long long warp_cnt[kWarps];  // packed counts per warp (see rank())
  unsigned long long warp_pre[kWarps];  // their exclusive prefix over warps
  unsigned long long tot;               // their totals
  unsigned long long s_acc[ACC_COUNT];
  uint64_t bar[2];
  TileInfo cur, next;
  int abort;
  float e_sec[kTile];  // energy handed to the secondary by an ionizing slot
};

__device__ __forceinline__ void set_error(Control* ctrl, int code) {
  atomicCAS(&ctrl->error, 0, code);
}

__device__ __forceinline__ void flush_segment(const DeviceRefs& r, int seg,
                                              unsigned long long* s_rho, CtaShared& cs,
                                              bool use_smem) {
  const int inst = seg >> 1, sp = seg & 1;
  const InstDev& P = r.inst[inst];
  __syncthreads();
  if (use_smem) {
    const int nn = P.n_cells + 1;
    unsigned long long* g = P.rho_acc[sp];
    for (int k = threadIdx.x; k < nn; k += kThreads) {
      const unsigned long long v = s_rho[k];
      if (v) {
        atomicAdd(g + k, v);
        s_rho[k] = 0ull;
      }
    }
  }
  if (threadIdx.x < ACC_COUNT) {
    const unsigned long long v = cs.s_acc[threadIdx.x];
    if (v) {
      atomicAdd(P.acc + threadIdx.x, v);
      cs.s_acc[threadIdx.x] = 0ull;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void deposit(unsigned long long* rho, int cell, float off,
                                        long long Q) {
  const long long right = right_share(Q, off);
  const long long left = Q - right;
  if (left) atomicAdd(rho + cell, (unsigned long long)left);
  if (right) atomicAdd(rho + cell + 1, (unsigned long long)right);
}

// Take the next tile (thread 0) and start its bulk loads into `stage`.
__device__ __forceinline__ TileInfo take_tile(const DeviceRefs& r, unsigned int n_tiles,
                                              float* stage, uint64_t* bar) {
  TileInfo t;
  t.g = atomicAdd(&r.ctrl->tile_counter, 1u);
  t.seg = -1;
  t.k = 0;
  t.fill = 0;
  if (t.g < n_tiles) {
    int lo = 0, hi = r.n_inst * 2 - 1;  // last segment with seg_start <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (r.seg_start[mid] <= t.g) lo = mid;
      else hi = mid - 1;
    }
    t.seg = lo;
    t.k = t.g - r.seg_start[lo];
    const SpeciesDev& S = r.inst[lo >> 1].sp[lo & 1];
    t.fill = S.fill[t.k];
    if (t.fill) {
      const SoA in = S.buf[r.sstate[lo].cur];
      const size_t base = (size_t)t.k * kTile;
      const uint32_t bytes = ((t.fill + 3u) & ~3u) * 4u;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(bar, 7u * bytes);
      bulk_load(stage + 0 * kTile, in.cell + base, bytes, bar);
      bulk_load(stage + 1 * kTile, in.off + base, bytes, bar);
      bulk_load(stage + 2 * kTile, in.vx + base, bytes, bar);
      bulk_load(stage + 3 * kTile, in.vy + base, bytes, bar);
      bulk_load(stage + 4 * kTile, in.vz + base, bytes, bar);
      bulk_load(stage + 5 * kTile, in.wj + base, bytes, bar);
      bulk_load(stage + 6 * kTile, in.id + base, bytes, bar);
    }
  }
  return t;
}

// ---- rare paths, kept out of line ----------------------------------------

struct Velocity {
  float vx, vy, vz;
};

// A null-collision candidate (u[0] < P0 already): choose the process with
// u[1] against the cumulative rates and scatter (Sec. IV).  Returns the new
// velocity; *proc_out = 0 elastic, 1 excitation, 2 ionization, 3 null.
__device__ __noinline__ Velocity collide(const InstDev& P, float kv, float vlim, float vx,
                                         float vy, float vz, float v1, float s1, uint4 rr,
                                         uint32_t id, uint32_t step, float wj,
                                         unsigned long long* acc, float* e_sec_out,
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

// A marker left the gap: tally the flux through the electrode (Eq. j); an ion
// at the cathode emits an electron with probability gamma.  Returns true when
// an electron is emitted.
__device__ __noinline__ bool absorb(const InstDev& P, int sp, int side, float wj, uint32_t id,
                                    uint32_t step, unsigned long long* acc) {
  const long long Qw = fixed_charge(wj, P.charge_shift);
  atomicAdd(&acc[ACC_NABS + sp * 2 + side], 1ull);
  atomicAdd(&acc[ACC_WABS + sp * 2 + side], (unsigned long long)Qw);
  if (sp != kIon || side != 0) return false;
  atomicAdd(&acc[ACC_WCATH], (unsigned long long)Qw);
  if (!(id & kGenBit)) atomicAdd(&acc[ACC_WCATH0], (unsigned long long)Qw);
  const uint4 rr =
      philox4x32_10(make_uint4(id, step, P.ctr_inst * 2u + 1u, 0u), P.key0, P.key1);
  if (!(uniform01(rr.x) < P.gamma)) return false;
  atomicAdd(&acc[ACC_SEE], 1ull);
  atomicAdd(&acc[ACC_WSEE], (unsigned long long)Qw);
  return true;
}

// Stage the electron and ion born by an ionization in slot o of the staging
// stores, and deposit both.
__device__ __noinline__ void stage_ionization(const InstDev& P, size_t o, int cell, float off,
                                              float wj, uint32_t id, uint32_t step, float es,
                                              unsigned long long* rho_e, bool smem_e) {
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
  deposit(rho_e, cell, off,
          fixed_charge(beta_of(sqrtf(bx * bx + by * by + bz * bz), SE.vlim) * wj,
                       P.charge_shift));
  (void)smem_e;
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

// Stage an electron emitted at the cathode (x = 0, at rest, the ion's w_j).
__device__ __noinline__ void stage_emission(const InstDev& P, size_t o, float wj) {
  const SpeciesDev& SE = P.sp[kElectron];
  SE.stage_b.cell[o] = 0;
  SE.stage_b.off[o] = 0.0f;
  SE.stage_b.vx[o] = 0.0f;
  SE.stage_b.vy[o] = 0.0f;
  SE.stage_b.vz[o] = 0.0f;
  SE.stage_b.wj[o] = wj;
  SE.stage_b.id[o] = kGenBit;
  // at rest: beta = 1, all the charge on node 0
  atomicAdd(P.rho_acc[kElectron], (unsigned long long)fixed_charge(wj, P.charge_shift));
}

// Field j (0..3) of a packed count word: 16 bits each.
__device__ __forceinline__ uint32_t field16(unsigned long long v, int j) {
  return (uint32_t)(v >> (16 * j)) & 0xFFFFu;
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 2) k_push(DeviceRefs r) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* stage0 = reinterpret_cast<float*>(smem_raw);
  float* stage1 = stage0 + 7 * kTile;
  unsigned long long* s_rho = reinterpret_cast<unsigned long long*>(stage1 + 7 * kTile);
  __shared__ CtaShared cs;

  Control* ctrl = r.ctrl;
  if (*((volatile int*)&ctrl->error)) return;
  const unsigned int n_tiles = ctrl->n_tiles;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lanemask_lt = (1u << lane) - 1u;

  for (int k = threadIdx.x; k < r.smem_nodes; k += kThreads) s_rho[k] = 0ull;
  if (threadIdx.x < ACC_COUNT) cs.s_acc[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) {
    mbar_init(&cs.bar[0], 1);
    mbar_init(&cs.bar[1], 1);
    fence_mbar_init();
    cs.abort = 0;
    cs.cur = take_tile(r, n_tiles, stage0, &cs.bar[0]);
  }
  __syncthreads();

  uint32_t phase0 = 0, phase1 = 0;
  int stage_idx = 0;
  int cur_seg = -1;
  bool use_smem = false;

  for (;;) {
    const TileInfo t = cs.cur;
    if (t.g >= n_tiles) break;
    float* st = stage_idx ? stage1 : stage0;
    int32_t* st_cell = reinterpret_cast<int32_t*>(st);
    float* st_off = st + 1 * kTile;
    float* st_vx = st + 2 * kTile;
    float* st_vy = st + 3 * kTile;
    float* st_vz = st + 4 * kTile;
    float* st_wj = st + 5 * kTile;
    uint32_t* st_id = reinterpret_cast<uint32_t*>(st + 6 * kTile);
    uint64_t* bar = &cs.bar[stage_idx];
    // prefetch the next tile into the other stage once the bulk stores that
    // read it (the previous tile) are done with it
    if (threadIdx.x == 0) {
      bulk_wait_read_all();
      cs.next = take_tile(r, n_tiles, stage_idx ? stage0 : stage1, &cs.bar[stage_idx ^ 1]);
    }
    if (t.seg != cur_seg) {
      if (cur_seg >= 0) flush_segment(r, cur_seg, s_rho, cs, use_smem);
      cur_seg = t.seg;
      use_smem = r.inst[t.seg >> 1].n_cells + 1 <= r.smem_nodes;
    }
    // wait for this tile's data (bounded)
    if (t.fill) {
      const uint32_t ph = stage_idx ? phase1 : phase0;
      uint32_t polls = 0;
      while (!mbar_try_wait(bar, ph)) {
        if (++polls > kSpinLimit) {
          set_error(ctrl, kErrTimeout);
          cs.abort = 1;
          break;
        }
      }
      if (threadIdx.x == 0 && polls) {
        atomicAdd(&ctrl->spin_waits, 1u);
        atomicMax(&ctrl->spin_max, polls);
      }
      if (stage_idx) phase1 ^= 1u;
      else phase0 ^= 1u;
    }

    const int inst = t.seg >> 1, sp = t.seg & 1;
    const InstDev& P = r.inst[inst];
    const SpeciesDev& S = P.sp[sp];
    const uint32_t step = r.istate[inst].step;
    unsigned long long* rho = use_smem ? s_rho : P.rho_acc[sp];
    const float qmdt = S.qmdt, vlim = S.vlim, kv = S.K_V, dtdx = P.dtdx, P0 = P.P0;
    const int N = P.n_cells, shift = P.charge_shift;
    const float* E32 = P.E32;
    const uint32_t key0 = P.key0, key1 = P.key1, ctr_e = P.ctr_inst * 2u;
    const bool electrons = sp == kElectron;

    // ---- 1. advance the thread's slots in place ------------------------------
    uint32_t alive_bits = 0, birth_bits = 0;
    uint32_t b_alive[kPerThread], b_birth[kPerThread];
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
      const int i = j * kThreads + threadIdx.x;
      bool alive = false, birth = false;
      if (i < (int)t.fill && !cs.abort) {
        int cell = st_cell[i];
        float off = st_off[i], vx = st_vx[i], vy = st_vy[i], vz = st_vz[i];
        // gather (linear between the cell's nodes)
        const float E0 = __ldg(E32 + cell), E1 = __ldg(E32 + cell + 1);
        const float Ex = E0 + off * (E1 - E0);
        // speed-limited kick (beta of the pre-kick speed) and drift (beta of
        // the post-kick speed)
        const float s0 = vx * vx + vy * vy + vz * vz;
        const float b0 = beta_of(sqrtf(s0), vlim);
        vx = vx + b0 * (qmdt * Ex);
        const float s1 = vx * vx + vy * vy + vz * vz;
        const float v1 = sqrtf(s1);
        float b1 = beta_of(v1, vlim);
        off = off + b1 * (vx * dtdx);
        const float fl = floorf(off);
        cell += (int)fl;
        off = off - fl;
        if (off >= 1.0f) {
          off = 0.0f;
          cell += 1;
        }
        if (cell < 0 || cell >= N) {
          birth = absorb(P, sp, cell < 0 ? 0 : 1, st_wj[i], st_id[i], step, cs.s_acc);
        } else {
          alive = true;
          const float wj = st_wj[i];
          if (electrons) {
            const uint32_t id = st_id[i];
            const uint4 rr = philox4x32_10(make_uint4(id, step, ctr_e, 0u), key0, key1);
            if (uniform01(rr.x) < P0) {
              int proc;
              float es = 0.0f;
              const Velocity nv = collide(P, kv, vlim, vx, vy, vz, v1, s1, rr, id, step, wj,
                                          cs.s_acc, &es, &proc);
              if (proc < 3) {
                vx = nv.vx;
                vy = nv.vy;
                vz = nv.vz;
                b1 = beta_of(sqrtf(vx * vx + vy * vy + vz * vz), vlim);
                st_vy[i] = vy;
                st_vz[i] = vz;
                if (proc == 2) {
                  birth = true;
                  cs.e_sec[i] = es;
                }
              }
            }
          }
          // deposit the survivor with w_p = beta w_j
          deposit(rho, cell, off, fixed_charge(b1 * wj, shift));
          st_cell[i] = cell;
          st_off[i] = off;
          st_vx[i] = vx;
        }
      }
      b_alive[j] = __ballot_sync(0xFFFFFFFFu, alive);
      b_birth[j] = __ballot_sync(0xFFFFFFFFu, birth);
      alive_bits |= (alive ? 1u : 0u) << j;
      birth_bits |= (birth ? 1u : 0u) << j;
    }

    // ---- 2. rank survivors and births inside the tile ------------------------
    // packed word: alive pass 0 | alive pass 1 | births pass 0 | births pass 1
    if (lane == 0) {
      cs.warp_cnt[warp] = (unsigned long long)__popc(b_alive[0]) |
                          ((unsigned long long)__popc(b_alive[1]) << 16) |
                          ((unsigned long long)__popc(b_birth[0]) << 32) |
                          ((unsigned long long)__popc(b_birth[1]) << 48);
    }
    __syncthreads();
    if (warp == 0) {
      const unsigned long long v = lane < kWarps ? cs.warp_cnt[lane] : 0ull;
      unsigned long long inc = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long n = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += n;
      }
      if (lane < kWarps) cs.warp_pre[lane] = inc - v;
      if (lane == kWarps - 1) cs.tot = inc;
    }
    __syncthreads();
    const unsigned long long pre = cs.warp_pre[warp], tot = cs.tot;
    const uint32_t n_surv = field16(tot, 0) + field16(tot, 1);
    const uint32_t n_birth = field16(tot, 2) + field16(tot, 3);

    // ---- 3. compact the survivors in place -----------------------------------
    int32_t c_cell[kPerThread];
    float c_off[kPerThread], c_vx[kPerThread], c_vy[kPerThread], c_vz[kPerThread],
        c_wj[kPerThread];
    uint32_t c_id[kPerThread];
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
      const int i = j * kThreads + threadIdx.x;
      if ((alive_bits | birth_bits) >> j & 1u) {
        c_cell[j] = st_cell[i];
        c_off[j] = st_off[i];
        c_vx[j] = st_vx[i];
        c_vy[j] = st_vy[i];
        c_vz[j] = st_vz[i];
        c_wj[j] = st_wj[i];
        c_id[j] = st_id[i];
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
      if (alive_bits >> j & 1u) {
        const uint32_t a = (j ? field16(tot, 0) : 0u) + field16(pre, j) +
                           (uint32_t)__popc(b_alive[j] & lanemask_lt);
        st_cell[a] = c_cell[j];
        st_off[a] = c_off[j];
        st_vx[a] = c_vx[j];
        st_vy[a] = c_vy[j];
        st_vz[a] = c_vz[j];
        st_wj[a] = c_wj[j];
        st_id[a] = c_id[j];
      }
    }
    fence_proxy_async_smem();
    __syncthreads();

    // ---- 4. store the compacted tile to its own slots ------------------------
    if (threadIdx.x == 0) {
      if (n_surv) {
        const SoA out = S.buf[r.sstate[t.seg].cur];
        const size_t base = (size_t)t.k * kTile;
        const uint32_t bytes = ((n_surv + 3u) & ~3u) * 4u;
        bulk_store(out.cell + base, st + 0 * kTile, bytes);
        bulk_store(out.off + base, st + 1 * kTile, bytes);
        bulk_store(out.vx + base, st + 2 * kTile, bytes);
        bulk_store(out.vy + base, st + 3 * kTile, bytes);
        bulk_store(out.vz + base, st + 4 * kTile, bytes);
        bulk_store(out.wj + base, st + 5 * kTile, bytes);
        bulk_store(out.id + base, st + 6 * kTile, bytes);
        bulk_commit();
      }
      if (t.g < n_tiles && t.seg >= 0) {
        S.fill[t.k] = n_surv;
        S.births[t.k] = n_birth;
      }
      atomicAdd(&cs.s_acc[ACC_MSTEPS], (unsigned long long)t.fill);
    }

    // ---- 5. births to tile-local staging slots -------------------------------
    if (birth_bits) {
      const size_t base = (size_t)t.k * kTile;
#pragma unroll
      for (int j = 0; j < kPerThread; ++j) {
        if (!(birth_bits >> j & 1u)) continue;
        const uint32_t b = (j ? field16(tot, 2) : 0u) + field16(pre, 2 + j) +
                           (uint32_t)__popc(b_birth[j] & lanemask_lt);
        if (electrons)
          stage_ionization(P, base + b, c_cell[j], c_off[j], c_wj[j], c_id[j], step,
                           cs.e_sec[j * kThreads + threadIdx.x], rho, use_smem);
        else
          stage_emission(P, base + b, c_wj[j]);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) cs.cur = cs.next;
    stage_idx ^= 1;
    __syncthreads();
    if (cs.abort) break;
  }
  if (cur_seg >= 0 && !cs.abort) flush_segment(r, cur_seg, s_rho, cs, use_smem);
  if (threadIdx.x == 0) {
    // no bulk copy may outlive the CTA's shared memory
    bulk_wait_all();
    if (cs.abort) {
      for (int s = 0; s < 2; ++s) {
        const uint32_t ph = s ? phase1 : phase0;
        for (uint32_t p = 0; p < kSpinLimit && !mbar_try_wait(&cs.bar[s], ph); ++p) {
        }
      }
    }
  }
}

int push_occupancy(int smem_nodes, int* blocks_per_sm, size_t* smem_bytes) {
  const size_t bytes = (size_t)2 * 7 * kTile * 4 + (size_t)smem_nodes * 8;
  cudaError_t e = cudaFuncSetAttribute(k_push, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return (int)e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_push, kThreads, bytes);
  *smem_bytes = bytes;
  return (int)e;
}

void launch_push(const DeviceRefs& r, int grid, cudaStream_t s) {
  const size_t bytes = (size_t)2 * 7 * kTile * 4 + (size_t)r.smem_nodes * 8;
  k_push<<<grid, kThreads, bytes, s>>>(r);
}

}  // namespace slpic
