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
//     advanced out of the other;
//   - each thread advances four consecutive markers in registers and
//     deposits the survivors into a shared-memory copy of the segment's charge
//     grid (integer atomics);
//   - a block scan ranks the survivors, which are written back compacted and
//     in order into the same stage and stored to the tile's own slots with bulk
//     copies; births go to tile-local staging slots.
// The shared charge grid is added to global memory with integer atomics when
// the CTA moves to another segment or finishes, so the deposit is exact and
// independent of the order of the additions.
#include "device_common.cuh"
#include "slpic_internal.h"

namespace slpic {

namespace {

struct Marker {
  int cell;
  float off, vx, vy, vz, wj;
  uint32_t id;
};

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
  unsigned long long warp_tot[kThreads / 32];
  unsigned long long s_acc[ACC_COUNT];
  uint64_t bar[2];
  TileInfo cur, next;
  int abort;
};

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long n = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// Exclusive block scan of packed counts (two 32-bit fields).
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v,
                                                              CtaShared& cs,
                                                              unsigned long long& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long inc = warp_incl_scan(v);
  if (lane == 31) cs.warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < kThreads / 32 ? cs.warp_tot[lane] : 0ull;
    w = warp_incl_scan(w);
    if (lane < kThreads / 32) cs.warp_tot[lane] = w;
  }
  __syncthreads();
  total = cs.warp_tot[kThreads / 32 - 1];
  const unsigned long long before = warp ? cs.warp_tot[warp - 1] : 0ull;
  return before + inc - v;
}

__device__ __forceinline__ void set_error(Control* ctrl, int code) {
  atomicCAS(&ctrl->error, 0, code);
}

__device__ __forceinline__ void flush_segment(const DeviceRefs& r, int seg,
                                              unsigned long long* s_rho, CtaShared& cs,
                                              long long wsurv, bool use_smem) {
  const int inst = seg >> 1, sp = seg & 1;
  const InstDev& P = r.inst[inst];
  long long w = wsurv;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xFFFFFFFFu, w, o);
  if ((threadIdx.x & 31) == 0 && w)
    atomicAdd(&cs.s_acc[ACC_WSURV + sp], (unsigned long long)w);
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

__device__ __forceinline__ void deposit(unsigned long long* s_rho, unsigned long long* g_rho,
                                        bool use_smem, int cell, float off, long long Q) {
  const long long right = right_share(Q, off);
  const long long left = Q - right;
  if (use_smem) {
    if (left) atomicAdd(s_rho + cell, (unsigned long long)left);
    if (right) atomicAdd(s_rho + cell + 1, (unsigned long long)right);
  } else {
    if (left) atomicAdd(g_rho + cell, (unsigned long long)left);
    if (right) atomicAdd(g_rho + cell + 1, (unsigned long long)right);
  }
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
  long long wsurv = 0;  // this thread's survivors' fixed-point weight, current segment

  for (;;) {
    const TileInfo t = cs.cur;
    if (t.g >= n_tiles) break;
    float* st = stage_idx ? stage1 : stage0;
    uint64_t* bar = &cs.bar[stage_idx];
    // prefetch the next tile into the other stage once the bulk stores that
    // read it (the previous tile) are done with it
    if (threadIdx.x == 0) {
      bulk_wait_read_all();
      cs.next = take_tile(r, n_tiles, stage_idx ? stage0 : stage1, &cs.bar[stage_idx ^ 1]);
    }
    if (t.seg != cur_seg) {
      if (cur_seg >= 0) flush_segment(r, cur_seg, s_rho, cs, wsurv, use_smem);
      wsurv = 0;
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
    __syncthreads();
    if (cs.abort) break;

    const int inst = t.seg >> 1, sp = t.seg & 1;
    const InstDev& P = r.inst[inst];
    const SpeciesDev& S = P.sp[sp];
    const uint32_t step = r.istate[inst].step;
    unsigned long long* g_rho = P.rho_acc[sp];
    const int i0 = threadIdx.x * kPerThread;

    // ---- 1. read four consecutive markers from the stage -------------------
    Marker m[kPerThread];
    const int nv = (int)t.fill - i0 < 0 ? 0 : min(kPerThread, (int)t.fill - i0);
    if (nv > 0) {
      const int4 c = *reinterpret_cast<const int4*>(st + 0 * kTile + i0);
      const float4 o = *reinterpret_cast<const float4*>(st + 1 * kTile + i0);
      const float4 x = *reinterpret_cast<const float4*>(st + 2 * kTile + i0);
      const float4 y = *reinterpret_cast<const float4*>(st + 3 * kTile + i0);
      const float4 z = *reinterpret_cast<const float4*>(st + 4 * kTile + i0);
      const float4 w = *reinterpret_cast<const float4*>(st + 5 * kTile + i0);
      const uint4 d = *reinterpret_cast<const uint4*>(st + 6 * kTile + i0);
      m[0] = {c.x, o.x, x.x, y.x, z.x, w.x, d.x};
      m[1] = {c.y, o.y, x.y, y.y, z.y, w.y, d.y};
      m[2] = {c.z, o.z, x.z, y.z, z.z, w.z, d.z};
      m[3] = {c.w, o.w, x.w, y.w, z.w, w.w, d.w};
    }

    // ---- 2. advance ----------------------------------------------------------
    const float qmdt = S.qmdt, vlim = S.vlim, dtdx = P.dtdx;
    const int N = P.n_cells;
    unsigned alive_mask = 0, birth_mask = 0;
    float e_sec[kPerThread];
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
      e_sec[k] = 0.0f;
      if (k >= nv) continue;
      Marker& q = m[k];
      // gather (linear between the cell's nodes)
      const float E0 = __ldg(P.E32 + q.cell), E1 = __ldg(P.E32 + q.cell + 1);
      const float Ex = E0 + q.off * (E1 - E0);
      // speed-limited kick (beta of the pre-kick speed) and drift (beta of
      // the post-kick speed)
      const float s0 = q.vx * q.vx + q.vy * q.vy + q.vz * q.vz;
      const float b0 = beta_of(sqrtf(s0), vlim);
      q.vx = q.vx + b0 * (qmdt * Ex);
      const float s1 = q.vx * q.vx + q.vy * q.vy + q.vz * q.vz;
      const float v1 = sqrtf(s1);
      float b1 = beta_of(v1, vlim);
      q.off = q.off + b1 * (q.vx * dtdx);
      const float fl = floorf(q.off);
      q.cell += (int)fl;
      q.off = q.off - fl;
      if (q.off >= 1.0f) {
        q.off = 0.0f;
        q.cell += 1;
      }
      // absorbing electrodes
      if (q.cell < 0 || q.cell >= N) {
        const int side = q.cell < 0 ? 0 : 1;
        const long long Qw = fixed_charge(q.wj, P.wscale);
        atomicAdd(&cs.s_acc[ACC_NABS + sp * 2 + side], 1ull);
        atomicAdd(&cs.s_acc[ACC_WABS + sp * 2 + side], (unsigned long long)Qw);
        if (sp == kIon && side == 0) {
          atomicAdd(&cs.s_acc[ACC_WCATH], (unsigned long long)Qw);
          if (!(q.id & kGenBit)) atomicAdd(&cs.s_acc[ACC_WCATH0], (unsigned long long)Qw);
          const uint4 rr = philox4x32_10(make_uint4(q.id, step, P.ctr_inst * 2u + 1u, 0u),
                                         P.key0, P.key1);
          if (uniform01(rr.x) < P.gamma) {
            birth_mask |= 1u << k;
            atomicAdd(&cs.s_acc[ACC_SEE], 1ull);
            atomicAdd(&cs.s_acc[ACC_WSEE], (unsigned long long)Qw);
          }
        }
        continue;
      }
      alive_mask |= 1u << k;
      if (sp == kElectron) {
        // null-collision test with the majorant probability P0
        const uint4 rr = philox4x32_10(make_uint4(q.id, step, P.ctr_inst * 2u, 0u), P.key0,
                                       P.key1);
        float u[4];
        uniform4(rr, u);
        if (u[0] < P.P0) {
          atomicAdd(&cs.s_acc[ACC_CAND], 1ull);
          float vb = v1 > vlim ? vlim : v1;
          if (vb > P.vb_cap) {
            vb = P.vb_cap;
            atomicAdd(&cs.s_acc[ACC_MAJ], 1ull);
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
          if (proc < 3) {
            atomicAdd(&cs.s_acc[ACC_COLL0 + proc], 1ull);
            if (proc == 0) {
              // Vahedi-Surendra: cos chi = (2 + eps - 2 (1 + eps)^u) / eps, with
              // 1 - cos chi and 1 + cos chi each formed without cancellation
              // so that sin chi keeps its relative precision at both ends
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
              float ux = q.vx / v1, uy = q.vy / v1, uz = q.vz / v1;
              rotate(ux, uy, uz, cc, sc, cp, sn);
              const float vn = sqrtf(e_new * S.K_V);
              q.vx = vn * ux;
              q.vy = vn * uy;
              q.vz = vn * uz;
            } else if (proc == 1) {
              float e_new = eps - P.e_ex;
              if (e_new < 0.0f) {
                e_new = 0.0f;
                atomicAdd(&cs.s_acc[ACC_CLAMP], 1ull);
              }
              isotropic(sqrtf(e_new * S.K_V), u[2], u[3], P.two_pi, q.vx, q.vy, q.vz);
            } else {
              float e_av = eps - P.e_io;
              if (e_av < 0.0f) {
                e_av = 0.0f;
                atomicAdd(&cs.s_acc[ACC_CLAMP], 1ull);
              }
              atomicAdd(&cs.s_acc[ACC_WIONZ],
                        (unsigned long long)fixed_charge(q.wj, P.wscale));
              const uint4 r1 = philox4x32_10(make_uint4(q.id, step, P.ctr_inst * 2u, 1u),
                                             P.key0, P.key1);
              const float es = uniform01(r1.x) * e_av;
              const float ep = e_av - es;
              isotropic(sqrtf(ep * S.K_V), u[2], u[3], P.two_pi, q.vx, q.vy, q.vz);
              e_sec[k] = es;
              birth_mask |= 1u << k;
            }
            b1 = beta_of(sqrtf(q.vx * q.vx + q.vy * q.vy + q.vz * q.vz), vlim);
          }
        }
      }
      // deposit the survivor with w_p = beta w_j
      const long long Q = fixed_charge(b1 * q.wj, P.wscale);
      deposit(s_rho, g_rho, use_smem, q.cell, q.off, Q);
      wsurv += fixed_charge(q.wj, P.wscale);
    }

    // ---- 3. rank survivors and births inside the tile ------------------------
    const unsigned long long packed = (unsigned long long)__popc(alive_mask) |
                                      ((unsigned long long)__popc(birth_mask) << 32);
    unsigned long long tot;
    const unsigned long long ex = block_excl_scan(packed, cs, tot);
    const unsigned int n_surv = (unsigned int)tot, n_birth = (unsigned int)(tot >> 32);
    // (the scan's barriers also order every read of the stage before the
    // compacted writes below)
    {
      unsigned int a = (unsigned int)ex;
#pragma unroll
      for (int k = 0; k < kPerThread; ++k) {
        if (alive_mask & (1u << k)) {
          reinterpret_cast<int32_t*>(st)[a] = m[k].cell;
          st[1 * kTile + a] = m[k].off;
          st[2 * kTile + a] = m[k].vx;
          st[3 * kTile + a] = m[k].vy;
          st[4 * kTile + a] = m[k].vz;
          st[5 * kTile + a] = m[k].wj;
          reinterpret_cast<uint32_t*>(st)[6 * kTile + a] = m[k].id;
          ++a;
        }
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
      S.fill[t.k] = n_surv;
      S.births[t.k] = n_birth;
      atomicAdd(&cs.s_acc[ACC_MSTEPS], (unsigned long long)t.fill);
    }

    // ---- 5. births to tile-local staging slots -------------------------------
    if (birth_mask) {
      unsigned int b = (unsigned int)(ex >> 32);
      const size_t base = (size_t)t.k * kTile;
      if (sp == kElectron) {
        const SpeciesDev& SI = P.sp[kIon];
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) {
          if (!(birth_mask & (1u << k))) continue;
          const Marker& q = m[k];
          const size_t o = base + b;
          const uint32_t gen = q.id & kGenBit;
          const uint4 r1 = philox4x32_10(make_uint4(q.id, step, P.ctr_inst * 2u, 1u), P.key0,
                                         P.key1);
          float bx, by, bz;
          isotropic(sqrtf(e_sec[k] * S.K_V), uniform01(r1.y), uniform01(r1.z), P.two_pi, bx,
                    by, bz);
          S.stage_a.cell[o] = q.cell;
          S.stage_a.off[o] = q.off;
          S.stage_a.vx[o] = bx;
          S.stage_a.vy[o] = by;
          S.stage_a.vz[o] = bz;
          S.stage_a.wj[o] = q.wj;
          S.stage_a.id[o] = gen;  // serial assigned when appended
          const long long Qe = fixed_charge(
              beta_of(sqrtf(bx * bx + by * by + bz * bz), vlim) * q.wj, P.wscale);
          deposit(s_rho, g_rho, use_smem, q.cell, q.off, Qe);
          // born ion: gas-temperature Maxwellian (Box-Muller on block 2)
          const uint4 r2 = philox4x32_10(make_uint4(q.id, step, P.ctr_inst * 2u, 2u), P.key0,
                                         P.key1);
          float gq[4];
          uniform4(r2, gq);
          const float rr1 = sqrtf(-2.0f * logf(gq[0]));
          const float rr2 = sqrtf(-2.0f * logf(gq[2]));
          const float a1 = P.two_pi * gq[1], a2 = P.two_pi * gq[3];
          const float ix = P.sigT_ion * (rr1 * cosf(a1));
          const float iy = P.sigT_ion * (rr1 * sinf(a1));
          const float iz = P.sigT_ion * (rr2 * cosf(a2));
          SI.stage_a.cell[o] = q.cell;
          SI.stage_a.off[o] = q.off;
          SI.stage_a.vx[o] = ix;
          SI.stage_a.vy[o] = iy;
          SI.stage_a.vz[o] = iz;
          SI.stage_a.wj[o] = q.wj;
          SI.stage_a.id[o] = gen;
          const long long Qi = fixed_charge(
              beta_of(sqrtf(ix * ix + iy * iy + iz * iz), SI.vlim) * q.wj, P.wscale);
          deposit(nullptr, P.rho_acc[kIon], false, q.cell, q.off, Qi);
          ++b;
        }
      } else {
        const SpeciesDev& SE = P.sp[kElectron];
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) {
          if (!(birth_mask & (1u << k))) continue;
          const size_t o = base + b;
          SE.stage_b.cell[o] = 0;
          SE.stage_b.off[o] = 0.0f;
          SE.stage_b.vx[o] = 0.0f;
          SE.stage_b.vy[o] = 0.0f;
          SE.stage_b.vz[o] = 0.0f;
          SE.stage_b.wj[o] = m[k].wj;
          SE.stage_b.id[o] = kGenBit;
          // emitted electron at rest at x = 0: beta = 1, all charge on node 0
          atomicAdd(P.rho_acc[kElectron],
                    (unsigned long long)fixed_charge(m[k].wj, P.wscale));
          ++b;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) cs.cur = cs.next;
    stage_idx ^= 1;
    __syncthreads();
  }
  if (cur_seg >= 0 && !cs.abort) flush_segment(r, cur_seg, s_rho, cs, wsurv, use_smem);
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
