// The particle kernel of one SLPIC-MCC step, batched over instances and
// species: gather, speed-limited kick and drift (Eqs. slpicEOMx, slpicEOMv,
// betaAbrupt), absorbing electrodes with ion-induced secondary emission
// (Sec. IV), null-collision Monte-Carlo collisions of electrons with a
// background gas (Sec. III, Eq. SLPICcollisionNumber with beta_n = 1),
// ionization births, stable compaction of survivors, and the fixed-point
// deposit of w_p = beta w_j (Eq. Ansatz).
//
// Work decomposition.  The markers of every (instance, species) segment are
// cut into tiles of kTile consecutive markers; a persistent grid takes tiles
// in increasing global order from an atomic counter.  Each tile:
//   1. loads its markers with 16-byte vector loads (SoA streams),
//   2. advances them in registers, depositing survivors into a shared-memory
//      copy of the segment's charge grid,
//   3. scans (survivor, ionization, emission) counts across the block,
//   4. obtains its exclusive prefix inside the segment by decoupled look-back
//      over the preceding tiles (bounded spins),
//   5. writes survivors compacted and in order to the other ping-pong buffer
//      through shared memory (coalesced stores), and births to staging.
// The shared charge grid is added to global memory with integer atomics when
// the CTA moves to another segment or finishes, so the deposit is exact and
// independent of the order of the additions.
#include <cuda/atomic>

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

// Per-tile scratch of the block scan and look-back.
struct TileShared {
  unsigned long long warp_tot[kThreads / 32];
  unsigned int prefix[3];
  unsigned int total[3];
  unsigned int tile;
  int seg;
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

// Exclusive block scan of packed counts (three 21-bit fields).
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v,
                                                              TileShared& ts,
                                                              unsigned long long& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long inc = warp_incl_scan(v);
  if (lane == 31) ts.warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < kThreads / 32 ? ts.warp_tot[lane] : 0ull;
    w = warp_incl_scan(w);
    if (lane < kThreads / 32) ts.warp_tot[lane] = w;
  }
  __syncthreads();
  total = ts.warp_tot[kThreads / 32 - 1];
  const unsigned long long before = warp ? ts.warp_tot[warp - 1] : 0ull;
  return before + inc - v;
}

constexpr unsigned long long kF1 = 1ull << 21, kF2 = 1ull << 42;
constexpr unsigned long long kFMask = (1ull << 21) - 1;

__device__ __forceinline__ void set_error(Control* ctrl, int code) {
  atomicCAS(&ctrl->error, 0, code);
}

__device__ __forceinline__ void flush_segment(const DeviceRefs& r, int seg,
                                              unsigned long long* s_rho,
                                              unsigned long long* s_acc, long long wsurv,
                                              bool use_smem) {
  const int inst = seg >> 1, sp = seg & 1;
  const InstDev& P = r.inst[inst];
  // survivors' weight: reduce the per-thread sums into the shared accumulators
  long long w = wsurv;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xFFFFFFFFu, w, o);
  if ((threadIdx.x & 31) == 0 && w) atomicAdd(&s_acc[ACC_WSURV + sp], (unsigned long long)w);
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
    const unsigned long long v = s_acc[threadIdx.x];
    if (v) {
      atomicAdd(P.acc + threadIdx.x, v);
      s_acc[threadIdx.x] = 0ull;
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

// Publish a look-back record: values first, then the flag with release order.
__device__ __forceinline__ void publish(TileStatus* t, const unsigned int v[3], bool inclusive,
                                        unsigned int epoch) {
  unsigned int* dst = inclusive ? t->incl : t->agg;
  dst[0] = v[0];
  dst[1] = v[1];
  dst[2] = v[2];
  cuda::atomic_ref<unsigned int, cuda::thread_scope_device> f(t->flag);
  f.store((epoch << 2) | (inclusive ? 2u : 1u), cuda::memory_order_release);
}

}  // namespace

__global__ void __launch_bounds__(kThreads) k_push(DeviceRefs r) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* s_rho = reinterpret_cast<unsigned long long*>(smem_raw);
  int32_t* s_cell = reinterpret_cast<int32_t*>(s_rho + r.smem_nodes);
  float* s_off = reinterpret_cast<float*>(s_cell + kTile);
  float* s_vx = s_off + kTile;
  float* s_vy = s_vx + kTile;
  float* s_vz = s_vy + kTile;
  float* s_wj = s_vz + kTile;
  uint32_t* s_id = reinterpret_cast<uint32_t*>(s_wj + kTile);
  __shared__ TileShared ts;
  __shared__ unsigned long long s_acc[ACC_COUNT];

  Control* ctrl = r.ctrl;
  if (*((volatile int*)&ctrl->error)) return;
  const unsigned int epoch = ctrl->epoch & 0x3FFFFFFFu;
  const unsigned int n_tiles = ctrl->n_tiles;
  const int n_seg = r.n_inst * 2;

  for (int k = threadIdx.x; k < r.smem_nodes; k += kThreads) s_rho[k] = 0ull;
  if (threadIdx.x < ACC_COUNT) s_acc[threadIdx.x] = 0ull;

  int cur_seg = -1;
  bool use_smem = false;
  long long wsurv = 0;  // this thread's survivors' fixed-point weight, current segment

  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned int g = atomicAdd(&ctrl->tile_counter, 1u);
      ts.tile = g;
      int seg = -1;
      if (g < n_tiles) {
        int lo = 0, hi = n_seg - 1;  // last segment with seg_start <= g
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (r.seg_start[mid] <= g) lo = mid;
          else hi = mid - 1;
        }
        seg = lo;
      }
      ts.seg = seg;
    }
    __syncthreads();
    const unsigned int g = ts.tile;
    const int seg = ts.seg;
    if (g >= n_tiles) break;
    if (seg != cur_seg) {
      if (cur_seg >= 0) flush_segment(r, cur_seg, s_rho, s_acc, wsurv, use_smem);
      wsurv = 0;
      cur_seg = seg;
      use_smem = r.inst[seg >> 1].n_cells + 1 <= r.smem_nodes;
    }
    const int inst = seg >> 1, sp = seg & 1;
    const InstDev& P = r.inst[inst];
    const SpeciesDev& S = P.sp[sp];
    SpeciesState* st = r.sstate + seg;
    const uint32_t cur = st->cur;
    const uint32_t n_live = st->n_live;
    const uint32_t step = r.istate[inst].step;
    const unsigned int lt = g - r.seg_start[seg];
    const uint32_t base = lt * kTile;
    const uint32_t i0 = base + threadIdx.x * kPerThread;
    const SoA in = S.buf[cur];
    const SoA out = S.buf[cur ^ 1u];
    unsigned long long* g_rho = P.rho_acc[sp];

    // ---- 1. load -------------------------------------------------------
    Marker m[kPerThread];
    int nv = 0;
    if (i0 + kPerThread <= n_live) {
      nv = kPerThread;
      const int4 c = __ldcs(reinterpret_cast<const int4*>(in.cell + i0));
      const float4 o = __ldcs(reinterpret_cast<const float4*>(in.off + i0));
      const float4 x = __ldcs(reinterpret_cast<const float4*>(in.vx + i0));
      const float4 y = __ldcs(reinterpret_cast<const float4*>(in.vy + i0));
      const float4 z = __ldcs(reinterpret_cast<const float4*>(in.vz + i0));
      const float4 w = __ldcs(reinterpret_cast<const float4*>(in.wj + i0));
      const uint4 d = __ldcs(reinterpret_cast<const uint4*>(in.id + i0));
      m[0] = {c.x, o.x, x.x, y.x, z.x, w.x, d.x};
      m[1] = {c.y, o.y, x.y, y.y, z.y, w.y, d.y};
      m[2] = {c.z, o.z, x.z, y.z, z.z, w.z, d.z};
      m[3] = {c.w, o.w, x.w, y.w, z.w, w.w, d.w};
    } else if (i0 < n_live) {
      nv = (int)(n_live - i0);
#pragma unroll
      for (int k = 0; k < kPerThread; ++k) {
        if (k < nv) {
          const uint32_t i = i0 + k;
          m[k] = {in.cell[i], in.off[i], in.vx[i], in.vy[i], in.vz[i], in.wj[i], in.id[i]};
        }
      }
    }

    // ---- 2. advance ----------------------------------------------------
    const float qmdt = S.qmdt, vlim = S.vlim, dtdx = P.dtdx;
    const int N = P.n_cells;
    unsigned alive_mask = 0, ionz_mask = 0, see_mask = 0;
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
        atomicAdd(&s_acc[ACC_NABS + sp * 2 + side], 1ull);
        atomicAdd(&s_acc[ACC_WABS + sp * 2 + side], (unsigned long long)Qw);
        if (sp == kIon && side == 0) {
          atomicAdd(&s_acc[ACC_WCATH], (unsigned long long)Qw);
          if (!(q.id & kGenBit)) atomicAdd(&s_acc[ACC_WCATH0], (unsigned long long)Qw);
          const uint4 rr = philox4x32_10(make_uint4(q.id, step, P.ctr_inst * 2u + 1u, 0u),
                                         P.key0, P.key1);
          if (uniform01(rr.x) < P.gamma) {
            see_mask |= 1u << k;
            atomicAdd(&s_acc[ACC_SEE], 1ull);
            atomicAdd(&s_acc[ACC_WSEE], (unsigned long long)Qw);
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
          atomicAdd(&s_acc[ACC_CAND], 1ull);
          float vb = v1 > vlim ? vlim : v1;
          if (vb > P.vb_cap) {
            vb = P.vb_cap;
            atomicAdd(&s_acc[ACC_MAJ], 1ull);
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
            atomicAdd(&s_acc[ACC_COLL0 + proc], 1ull);
            if (proc == 0) {
              // Vahedi-Surendra: cos chi = 1 - 2 expm1(u log1p(eps)) / eps
              const float em = expm1f(u[2] * log1pf(eps));
              float cc = 1.0f - (em + em) / eps;
              cc = fminf(1.0f, fmaxf(-1.0f, cc));
              const float sc = sqrtf(fmaxf(0.0f, (1.0f - cc) * (1.0f + cc)));
              const float ph = P.two_pi * u[3];
              const float cp = cosf(ph), sn = sinf(ph);
              const float e_new = eps * (1.0f - P.R2 * (1.0f - cc));
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
                atomicAdd(&s_acc[ACC_CLAMP], 1ull);
              }
              isotropic(sqrtf(e_new * S.K_V), u[2], u[3], P.two_pi, q.vx, q.vy, q.vz);
            } else {
              float e_av = eps - P.e_io;
              if (e_av < 0.0f) {
                e_av = 0.0f;
                atomicAdd(&s_acc[ACC_CLAMP], 1ull);
              }
              atomicAdd(&s_acc[ACC_WIONZ], (unsigned long long)fixed_charge(q.wj, P.wscale));
              const uint4 r1 = philox4x32_10(make_uint4(q.id, step, P.ctr_inst * 2u, 1u),
                                             P.key0, P.key1);
              const float es = uniform01(r1.x) * e_av;
              const float ep = e_av - es;
              isotropic(sqrtf(ep * S.K_V), u[2], u[3], P.two_pi, q.vx, q.vy, q.vz);
              e_sec[k] = es;
              ionz_mask |= 1u << k;
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

    // ---- 3. block scan of the counts ------------------------------------
    const unsigned long long packed = (unsigned long long)__popc(alive_mask) |
                                      ((unsigned long long)__popc(ionz_mask) << 21) |
                                      ((unsigned long long)__popc(see_mask) << 42);
    unsigned long long tot;
    const unsigned long long ex = block_excl_scan(packed, ts, tot);
    const unsigned int ra = (unsigned int)(ex & kFMask);
    const unsigned int rb = (unsigned int)((ex >> 21) & kFMask);
    const unsigned int rc = (unsigned int)((ex >> 42) & kFMask);
    // stage survivors in shared memory at their rank inside the tile
    {
      unsigned int a = ra;
#pragma unroll
      for (int k = 0; k < kPerThread; ++k) {
        if (alive_mask & (1u << k)) {
          s_cell[a] = m[k].cell;
          s_off[a] = m[k].off;
          s_vx[a] = m[k].vx;
          s_vy[a] = m[k].vy;
          s_vz[a] = m[k].vz;
          s_wj[a] = m[k].wj;
          s_id[a] = m[k].id;
          ++a;
        }
      }
    }

    // ---- 4. decoupled look-back ------------------------------------------
    if (threadIdx.x == 0) {
      const unsigned int agg[3] = {(unsigned int)(tot & kFMask),
                                   (unsigned int)((tot >> 21) & kFMask),
                                   (unsigned int)((tot >> 42) & kFMask)};
      TileStatus* t = r.tiles + g;
      unsigned int excl[3] = {0u, 0u, 0u};
      if (lt == 0) {
        publish(t, agg, true, epoch);
      } else {
        publish(t, agg, false, epoch);
        unsigned int j = g - 1;
        bool timed_out = false;
        for (;;) {
          cuda::atomic_ref<unsigned int, cuda::thread_scope_device> f(r.tiles[j].flag);
          unsigned int fv = f.load(cuda::memory_order_acquire);
          uint32_t spins = 0;
          while ((fv >> 2) != epoch || (fv & 3u) == 0u) {
            if (++spins > kSpinLimit || *((volatile int*)&ctrl->error) == kErrTimeout) {
              timed_out = true;
              break;
            }
            __nanosleep(64);
            fv = f.load(cuda::memory_order_acquire);
          }
          if (timed_out) {
            set_error(ctrl, kErrTimeout);
            break;
          }
          const volatile unsigned int* v =
              (fv & 3u) == 2u ? r.tiles[j].incl : r.tiles[j].agg;
          excl[0] += v[0];
          excl[1] += v[1];
          excl[2] += v[2];
          if ((fv & 3u) == 2u) break;
          --j;
        }
        const unsigned int incl[3] = {excl[0] + agg[0], excl[1] + agg[1], excl[2] + agg[2]};
        publish(t, incl, true, epoch);
      }
      ts.prefix[0] = excl[0];
      ts.prefix[1] = excl[1];
      ts.prefix[2] = excl[2];
      ts.total[0] = agg[0];
      ts.total[1] = agg[1];
      ts.total[2] = agg[2];
      // the segment's last tile records the segment's totals
      if (g + 1 == r.seg_start[seg + 1]) {
        st->n_surv = excl[0] + agg[0];
        if (sp == kElectron) {
          st->n_ba = excl[1] + agg[1];
          r.sstate[seg + 1].n_ba = excl[1] + agg[1];
        } else {
          r.sstate[seg - 1].n_bb = excl[2] + agg[2];
        }
      }
      atomicAdd(&s_acc[ACC_MSTEPS], (unsigned long long)min((uint32_t)kTile, n_live - base));
    }
    __syncthreads();

    // ---- 5. write survivors and births -----------------------------------
    const unsigned int pa = ts.prefix[0], na = ts.total[0];
    for (unsigned int i = threadIdx.x; i < na; i += kThreads) {
      const unsigned int o = pa + i;
      __stcs(out.cell + o, s_cell[i]);
      __stcs(out.off + o, s_off[i]);
      __stcs(out.vx + o, s_vx[i]);
      __stcs(out.vy + o, s_vy[i]);
      __stcs(out.vz + o, s_vz[i]);
      __stcs(out.wj + o, s_wj[i]);
      __stcs(out.id + o, s_id[i]);
    }
    if (ionz_mask) {
      const SpeciesDev& SI = P.sp[kIon];
      const uint32_t next_e = st->next_id, next_i = r.sstate[seg + 1].next_id;
      unsigned int b = ts.prefix[1] + rb;
#pragma unroll
      for (int k = 0; k < kPerThread; ++k) {
        if (!(ionz_mask & (1u << k))) continue;
        const Marker& q = m[k];
        if (b >= S.stage_cap || b >= SI.stage_cap) {
          set_error(ctrl, kErrCapacity);
          ++b;
          continue;
        }
        if (next_e + b > kSerialMask || next_i + b > kSerialMask) set_error(ctrl, kErrIdWrap);
        const uint32_t gen = q.id & kGenBit;
        const uint4 r1 = philox4x32_10(make_uint4(q.id, step, P.ctr_inst * 2u, 1u), P.key0,
                                       P.key1);
        float bx, by, bz;
        isotropic(sqrtf(e_sec[k] * S.K_V), uniform01(r1.y), uniform01(r1.z), P.two_pi, bx,
                  by, bz);
        S.stage_a.cell[b] = q.cell;
        S.stage_a.off[b] = q.off;
        S.stage_a.vx[b] = bx;
        S.stage_a.vy[b] = by;
        S.stage_a.vz[b] = bz;
        S.stage_a.wj[b] = q.wj;
        S.stage_a.id[b] = gen | ((next_e + b) & kSerialMask);
        const long long Qe =
            fixed_charge(beta_of(sqrtf(bx * bx + by * by + bz * bz), vlim) * q.wj, P.wscale);
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
        SI.stage_a.cell[b] = q.cell;
        SI.stage_a.off[b] = q.off;
        SI.stage_a.vx[b] = ix;
        SI.stage_a.vy[b] = iy;
        SI.stage_a.vz[b] = iz;
        SI.stage_a.wj[b] = q.wj;
        SI.stage_a.id[b] = gen | ((next_i + b) & kSerialMask);
        const long long Qi = fixed_charge(
            beta_of(sqrtf(ix * ix + iy * iy + iz * iz), SI.vlim) * q.wj, P.wscale);
        deposit(nullptr, P.rho_acc[kIon], false, q.cell, q.off, Qi);
        ++b;
      }
    }
    if (see_mask) {
      const SpeciesDev& SE = P.sp[kElectron];
      unsigned int b = ts.prefix[2] + rc;
#pragma unroll
      for (int k = 0; k < kPerThread; ++k) {
        if (!(see_mask & (1u << k))) continue;
        if (b >= SE.stage_cap) {
          set_error(ctrl, kErrCapacity);
          ++b;
          continue;
        }
        SE.stage_b.cell[b] = 0;
        SE.stage_b.off[b] = 0.0f;
        SE.stage_b.vx[b] = 0.0f;
        SE.stage_b.vy[b] = 0.0f;
        SE.stage_b.vz[b] = 0.0f;
        SE.stage_b.wj[b] = m[k].wj;
        SE.stage_b.id[b] = kGenBit;  // serial assigned when appended
        // emitted electron at rest at x = 0: beta = 1, all charge on node 0
        atomicAdd(P.rho_acc[kElectron], (unsigned long long)fixed_charge(m[k].wj, P.wscale));
        ++b;
      }
    }
    __syncthreads();
  }
  if (cur_seg >= 0) flush_segment(r, cur_seg, s_rho, s_acc, wsurv, use_smem);
}

int push_occupancy(int smem_nodes, int* blocks_per_sm, size_t* smem_bytes) {
  const size_t bytes = (size_t)smem_nodes * 8 + (size_t)kTile * 7 * 4;
  cudaError_t e = cudaFuncSetAttribute(k_push, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return (int)e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_push, kThreads, bytes);
  *smem_bytes = bytes;
  return (int)e;
}

void launch_push(const DeviceRefs& r, int grid, cudaStream_t s) {
  const size_t bytes = (size_t)r.smem_nodes * 8 + (size_t)kTile * 7 * 4;
  k_push<<<grid, kThreads, bytes, s>>>(r);
}

}  // namespace slpic
