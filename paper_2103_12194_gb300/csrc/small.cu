// Whole steps of small populations in one launch.  The paper's own runs
// start from 100 electrons at rest and stay at hundreds to thousands of
// markers near breakdown (Sec. V), where a step of the batched kernels is
// bound by its four launches and their grid-wide hand-offs, not by the
// markers.  Here one CTA of 512 threads owns one instance and runs the
// steps back to back with block barriers only:
//   1. push: warp w advances tiles w, w + 16, ... of both species with the
//      same arithmetic as the particle kernel (gather, speed-limited kick and
//      drift, electrodes and emission, the candidate draw, in-tile
//      compaction), straight from global memory;
//   2. collisions: thread t takes candidates t, t + 512, ... in (tile, slot)
//      order; the births get their slots from one block scan (ionization
//      pairs in candidate order, then the emitted electrons in ion-tile
//      order), exactly the order of the batched path;
//   3. finish: counts and fills, repacking of a sparse store, the deposit of
//      every live marker, the Poisson solve (field mode 1) and the step's
//      tallies.
// The deposit of a step is a function of the markers after it (each live
// marker adds fixed_charge(beta(|v|) w_j) at its position), so it is formed
// in one pass at the end of the step, into shared memory; with an imposed
// field nothing reads it during the run, and it is formed when it is read.
// With several instances, every CTA waits at a grid barrier before each
// step (a cooperative launch keeps them resident), so that all stop at the
// same step when one store outgrows the path; the host then continues with
// the batched kernels.  Results equal the batched path's bit for bit.
#include "device_common.cuh"
#include "slpic_internal.h"
#include "step_ops.cuh"

namespace slpic {

namespace {

constexpr int kSmallThreads = 512;
constexpr int kSmallWarps = kSmallThreads / 32;
// Tiles a store can reach in one step from at most kSmallMaxTiles tiles of
// each species: electrons double at most and gain one emitted electron per
// ion; ions gain one per electron.
constexpr int kSmallFillCap = 4 * kSmallMaxTiles;
constexpr int kSmallCandRows = kSmallMaxTiles * kTile / kSmallThreads;
static_assert(kSmallMaxTiles <= 32, "one lane per tile in the prefix scans");
static_assert(kSmallCandRows * kSmallThreads == kSmallMaxTiles * kTile, "candidate rows");
static_assert(kSmallCandRows <= 8, "16-bit row counters in one 128-bit scan value");

struct SmallShared {
  unsigned long long acc[ACC_COUNT];
  uint32_t fill[2][kSmallFillCap];
  uint32_t cnt[2][kSmallMaxTiles];  // per tile: candidates (electrons), emissions (ions)
  uint32_t pre[2][kSmallFillCap];   // exclusive prefixes (counts; fills when repacking)
  uint32_t tot[2];
  SpeciesState st[2];
  uint32_t tail[2], end[2], n_new[2], nt[2], nb[2], compact[2];
  uint32_t step;
  long long n_steps_done;
  unsigned long long w_live[2];
  long long ion_steps;
  long long i64[32];
  __int128 i128[32];
  int stop;
};

// Last tile j < n whose exclusive prefix pre[j] is at or below e (that tile
// holds event e).
__device__ __forceinline__ int tile_of_event(const uint32_t* pre, int n, uint32_t e) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Deposit of every live marker of instance P after a step into rho[sp]
// (nn nodes per species): w_p = beta(|v|) w_j in fixed point at the marker's
// position, as each marker was deposited by the batched path.
template <typename R>
__device__ void deposit_all(const InstDev& P, const SmallShared& sh, unsigned long long* rho0,
                            unsigned long long* rho1) {
  const StepConsts<R>& K = consts<R>(P);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ne = (int)sh.st[0].n_tiles, n_items = ne + (int)sh.st[1].n_tiles;
  for (int it = warp; it < n_items; it += kSmallWarps) {
    const int sp = it < ne ? 0 : 1, k = it < ne ? it : it - ne;
    const SoAT<R> m = soa_as<R>(P.sp[sp].buf[sh.st[sp].cur]);
    const R vlim = K.vlim[sp];
    const bool limited = vlim < (R)INFINITY;
    unsigned long long* rho = sp ? rho1 : rho0;
    const uint32_t n = sh.fill[sp][k];
    const size_t base = (size_t)k * kTile;
    for (uint32_t i = lane; i < n; i += 32) {
      const size_t o = base + i;
      const R vx = m.vx[o], vy = m.vy[o], vz = m.vz[o];
      const R b = limited ? beta_of(r_sqrt(vx * vx + vy * vy + vz * vz), vlim) : (R)1;
      deposit(rho, m.cell[o], m.off[o], fixed_charge(b * m.wj[o], K.wscale));
    }
  }
}

// Exclusive prefix of v[0 .. n) (n <= 4 * 32) by one warp into pre; returns
// the total.
__device__ __forceinline__ uint32_t warp_prefix(const uint32_t* v, int n, uint32_t* pre) {
  const int lane = threadIdx.x & 31;
  uint32_t loc[4], sum = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int k = lane * 4 + j;
    loc[j] = k < n ? v[k] : 0u;
    sum += loc[j];
  }
  uint32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += y;
  }
  uint32_t run = inc - sum;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int k = lane * 4 + j;
    if (k < n) pre[k] = run;
    run += loc[j];
  }
  return __shfl_sync(0xFFFFFFFFu, inc, 31);
}

}  // namespace

// Up to n_steps steps of instance blockIdx.x; stops before a step when a
// store of any instance has more than max_tiles tiles, or on a device error.
// Dynamic shared memory (field mode 1): two int64 deposit grids and the FP64
// node field, (N + 1) nodes each.
template <typename R>
__global__ void __launch_bounds__(kSmallThreads, 1) k_small(DeviceRefs r, long long n_steps,
                                                            int max_tiles) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ SmallShared sh;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint32_t lanemask_lt = (1u << lane) - 1u;
  Control* ctrl = r.ctrl;
  const int inst = blockIdx.x;
  const InstDev& P = r.inst[inst];
  InstState& gis = r.istate[inst];
  const StepConsts<R>& K = consts<R>(P);
  const int N = P.n_cells, nn = N + 1;
  const bool poisson = P.field_mode == 1;
  unsigned long long* s_rho0 = reinterpret_cast<unsigned long long*>(s_dyn);
  unsigned long long* s_rho1 = s_rho0 + nn;
  double* s_E = reinterpret_cast<double*>(s_rho1 + nn);
  const SpeciesDev& E = P.sp[kElectron];
  const SpeciesDev& I = P.sp[kIon];

  // ---- the instance's state into shared memory --------------------------------
  if (t < 2) sh.st[t] = r.sstate[inst * 2 + t];
  if (t < ACC_COUNT) sh.acc[t] = 0ull;
  if (t == 0) {
    sh.step = gis.step;
    sh.n_steps_done = gis.n_steps_done;
    sh.w_live[0] = gis.w_live[0];
    sh.w_live[1] = gis.w_live[1];
    sh.ion_steps = gis.ion_steps;
  }
  __syncthreads();
  for (int sp = 0; sp < 2; ++sp) {
    const uint32_t n = min(sh.st[sp].n_tiles, (uint32_t)kSmallFillCap);
    for (uint32_t k = t; k < n; k += kSmallThreads) sh.fill[sp][k] = P.sp[sp].fill[sh.st[sp].cur][k];
  }
  if (poisson) {
    for (int k = t; k < nn; k += kSmallThreads) {
      s_rho0[k] = 0ull;
      s_rho1[k] = 0ull;
      s_E[k] = P.E64[k];
    }
  }
  const R* Eglob = node_field<R>(P);

  long long done = 0;
  for (;;) {
    // ---- another step? all CTAs decide together ------------------------------
    __syncthreads();
    if (t == 0) {
      int stop = done >= n_steps ? 2 : 0;
      if (!stop && ((int)sh.st[0].n_tiles > max_tiles || (int)sh.st[1].n_tiles > max_tiles ||
                    *((volatile int*)&ctrl->error)))
        stop = 1;
      if (stop != 2 && gridDim.x > 1) {
        // grid barrier b = done: arrive, then wait (bounded) for every CTA
        if (stop) atomicOr(&ctrl->small_stop, 1);
        __threadfence();
        // test hook: one CTA leaves out its arrival at one barrier, so that
        // every CTA's bounded wait there runs out (its own included)
        const bool skip = *((volatile int*)&ctrl->skip_cta) == (int)blockIdx.x + 1 &&
                          *((volatile long long*)&ctrl->skip_barrier) == done + 1;
        if (skip) *((volatile int*)&ctrl->skip_cta) = 0;  // once
        else atomicAdd(&ctrl->small_bar, 1u);
        const unsigned int target = (unsigned int)(done + 1) * gridDim.x;
        const uint32_t limit = spin_limit(ctrl);
        uint32_t polls = 0;
        while (*((volatile unsigned int*)&ctrl->small_bar) < target) {
          if (++polls > limit) {
            atomicCAS(&ctrl->error, 0, kErrTimeout);
            stop = 1;
            break;
          }
          __nanosleep(64);
        }
        __threadfence();
        if (*((volatile int*)&ctrl->small_stop)) stop = 1;
      }
      sh.stop = stop;
    }
    __syncthreads();
    if (sh.stop) break;
    const uint32_t step = sh.step;

    // ---- 1. push: one warp per tile ---------------------------------------------
    {
      const int ne = (int)sh.st[0].n_tiles, n_items = ne + (int)sh.st[1].n_tiles;
      for (int it = warp; it < n_items; it += kSmallWarps) {
        const int sp = it < ne ? 0 : 1, kt = it < ne ? it : it - ne;
        const SpeciesDev& S = P.sp[sp];
        const SoAT<R> m = soa_as<R>(S.buf[sh.st[sp].cur]);
        const uint32_t fill = sh.fill[sp][kt];
        const size_t tbase = (size_t)kt * kTile;
        uint32_t n_surv = 0, n_event = 0;
        int cell[kPerLane];
        R off[kPerLane], vx[kPerLane], vy[kPerLane], vz[kPerLane], wj[kPerLane];
        uint32_t id[kPerLane];
        bool live[kPerLane];
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) {
          const int i = j * 32 + lane;
          live[j] = i < (int)fill;
          const size_t o = tbase + i;
          cell[j] = live[j] ? m.cell[o] : 0;
          off[j] = live[j] ? m.off[o] : (R)0;
          vx[j] = live[j] ? m.vx[o] : (R)0;
          vy[j] = live[j] ? m.vy[o] : (R)0;
          vz[j] = live[j] ? m.vz[o] : (R)0;
          wj[j] = live[j] ? m.wj[o] : (R)0;
          id[j] = live[j] ? m.id[o] : 0u;
        }
        const R qmdt = K.qmdt[sp], vlim = K.vlim[sp], dtdx = K.dtdx, P0 = K.P0;
        const uint32_t Nc = (uint32_t)N;
        const bool electrons = sp == kElectron;
        const bool limited = vlim < (R)INFINITY;
        R a[kPerLane], b1[kPerLane];
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) {
          R E0, E1;
          if (poisson) {
            E0 = (R)s_E[cell[j]];
            E1 = (R)s_E[cell[j] + 1];
          } else {
            E0 = __ldg(Eglob + cell[j]);
            E1 = __ldg(Eglob + cell[j] + 1);
          }
          a[j] = qmdt * (E0 + off[j] * (E1 - E0));
        }
        if (limited) {
          limited_kick_n<R, kPerLane>(vx, vy, vz, a, vlim);
#pragma unroll
          for (int j = 0; j < kPerLane; ++j)
            b1[j] = beta_of(r_sqrt(vx[j] * vx[j] + vy[j] * vy[j] + vz[j] * vz[j]), vlim);
        } else {
#pragma unroll
          for (int j = 0; j < kPerLane; ++j) {
            vx[j] = vx[j] + a[j];
            b1[j] = (R)1;
          }
        }
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) {
          R o = off[j] + b1[j] * (vx[j] * dtdx);
          const R fl = r_floor(o);
          int c = cell[j] + (int)fl;
          o = o - fl;
          if (o >= (R)1) {
            o = (R)0;
            c += 1;
          }
          cell[j] = c;
          off[j] = o;
        }
        bool alive[kPerLane], event[kPerLane];
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) {
          alive[j] = live[j] && (uint32_t)cell[j] < Nc;
          event[j] = false;
        }
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) {
          if (live[j] && !alive[j])
            event[j] = absorb<R>(P, sp, cell[j] < 0 ? 0 : 1, wj[j], id[j], step, sh.acc, vx[j],
                                 vy[j], vz[j]);
        }
        if (electrons) {
          const uint32_t key2 = P.key2;
#pragma unroll
          for (int j = 0; j < kPerLane; ++j) {
            const uint2 rr = philox2x32_10(make_uint2(id[j], step), key2);
            event[j] = alive[j] && uniform01r<R>(rr.x) < P0;
          }
        }
        uint32_t b_alive[kPerLane], b_event[kPerLane];
        uint32_t pre_alive[kPerLane], pre_event[kPerLane];
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) {
          b_alive[j] = __ballot_sync(0xFFFFFFFFu, alive[j]);
          b_event[j] = __ballot_sync(0xFFFFFFFFu, event[j]);
          pre_alive[j] = n_surv;
          pre_event[j] = n_event;
          n_surv += __popc(b_alive[j]);
          n_event += __popc(b_event[j]);
        }
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) {
          if (event[j]) {
            const uint32_t e = pre_event[j] + (uint32_t)__popc(b_event[j] & lanemask_lt);
            if (electrons) {
              const uint32_t r_a = pre_alive[j] + (uint32_t)__popc(b_alive[j] & lanemask_lt);
              put_cand(S.crec, tbase + e, cell[j], off[j], vx[j], vy[j], vz[j], wj[j], id[j],
                       r_a);
            } else {
              stage_emission<R, false>(P, tbase + e, wj[j]);
            }
          }
        }
        // survivors back to the tile's own slots, compacted in order when a
        // marker left (every lane read its slots above)
        __syncwarp();
        const bool compact = n_surv != fill;
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) {
          if (!alive[j]) continue;
          if (!compact) {
            const size_t o = tbase + j * 32 + lane;
            m.cell[o] = cell[j];
            m.off[o] = off[j];
            m.vx[o] = vx[j];
          } else {
            const size_t o =
                tbase + pre_alive[j] + (uint32_t)__popc(b_alive[j] & lanemask_lt);
            m.cell[o] = cell[j];
            m.off[o] = off[j];
            m.vx[o] = vx[j];
            m.vy[o] = vy[j];
            m.vz[o] = vz[j];
            m.wj[o] = wj[j];
            m.id[o] = id[j];
          }
        }
        if (lane == 0) {
          sh.fill[sp][kt] = n_surv;
          sh.cnt[sp][kt] = n_event;
          if (fill) atomicAdd(&sh.acc[ACC_MSTEPS], (unsigned long long)fill);
        }
      }
    }
    __syncthreads();

    // ---- 2. collisions and births ---------------------------------------------
    if (warp < 2) {
      const uint32_t tot = warp_prefix(sh.cnt[warp], (int)sh.st[warp].n_tiles, sh.pre[warp]);
      if (lane == 0) sh.tot[warp] = tot;
    }
    __syncthreads();
    const SpeciesState se = sh.st[0], si = sh.st[1];
    const SoAT<R> me = soa_as<R>(E.buf[se.cur]);
    const SoAT<R> mi = soa_as<R>(I.buf[si.cur]);
    const uint32_t app_e = se.n_tiles ? (se.n_tiles - 1) * (uint32_t)kTile + sh.fill[0][se.n_tiles - 1] : 0u;
    const uint32_t app_i = si.n_tiles ? (si.n_tiles - 1) * (uint32_t)kTile + sh.fill[1][si.n_tiles - 1] : 0u;
    const uint32_t cap_e = E.cap_tiles * (uint32_t)kTile, cap_i = I.cap_tiles * (uint32_t)kTile;
    {
      const uint32_t C = sh.tot[0];
      const R kv = K.K_V[kElectron], vlim = K.vlim[kElectron];
      uint32_t slot[kSmallCandRows];
      R es[kSmallCandRows];
      unsigned __int128 flags = 0;  // 16-bit ionization count per row
      uint32_t n_proc[3] = {0u, 0u, 0u};  // this thread's collisions by kind
#pragma unroll
      for (int u = 0; u < kSmallCandRows; ++u) {
        const uint32_t c = (uint32_t)t + (uint32_t)u * kSmallThreads;
        slot[u] = 0u;
        es[u] = (R)0;
        if (c >= C) continue;
        const int j = tile_of_event(sh.pre[0], (int)se.n_tiles, c);
        const uint32_t q = c - sh.pre[0][j];
        const size_t base = (size_t)j * kTile;
        const CandRec<R> cr = get_cand<R>(E.crec, base + q);
        const size_t o = base + cr.slot;
        slot[u] = (uint32_t)o;
        const uint32_t id = cr.id;
        R vx = cr.vx, vy = cr.vy, vz = cr.vz;
        const R s1 = vx * vx + vy * vy + vz * vz;
        const R v1 = r_sqrt(s1);
        const uint4 rr = philox4x32_10(make_uint4(id, step, P.ctr_inst * 2u, 0u), P.key0, P.key1);
        int proc;
        R e2 = (R)0;
        const Velocity<R> nv = collide<R>(P, kv, vlim, vx, vy, vz, v1, s1, rr, id, step,
                                          cr.wj, sh.acc, &e2, &proc);
        if (proc < 3) ++n_proc[proc];
        if (proc < 3) {
          me.vx[o] = nv.vx;
          me.vy[o] = nv.vy;
          me.vz[o] = nv.vz;
          if (proc == 2) {
            flags |= (unsigned __int128)1 << (16 * u);
            es[u] = e2;
          }
        }
      }
      // the step's candidates and collisions, counted once per warp (C by
      // one thread) instead of an atomic per candidate on shared counters
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const uint32_t nw = __reduce_add_sync(0xFFFFFFFFu, n_proc[k]);
        if ((t & 31) == 0 && nw) atomicAdd(&sh.acc[ACC_COLL0 + k], (unsigned long long)nw);
      }
      if (t == 0 && C) atomicAdd(&sh.acc[ACC_CAND], (unsigned long long)C);
      // ranks of the ionizations in candidate order: c = t + kSmallThreads u,
      // so row u precedes row u + 1 and inside a row the threads are in order
      // (the scan is skipped in the many steps without an ionization)
      unsigned __int128 incl = 0, rows = 0;
      if (__syncthreads_or(flags != 0)) {
        incl = (unsigned __int128)block_incl_scan<__int128, kSmallThreads>((__int128)flags,
                                                                           sh.i128);
        if (t == kSmallThreads - 1) sh.i128[0] = (__int128)incl;  // row totals
        __syncthreads();
        rows = (unsigned __int128)sh.i128[0];
        __syncthreads();
      }
      const unsigned __int128 excl = incl - flags;
      uint32_t before = 0;  // ionizations in the rows above
#pragma unroll
      for (int u = 0; u < kSmallCandRows; ++u) {
        if ((uint32_t)(flags >> (16 * u)) & 1u) {
          const uint32_t rank = before + ((uint32_t)(excl >> (16 * u)) & 0xFFFFu);
          const uint32_t pe = app_e + rank, pi = app_i + rank;
          const uint32_t o = slot[u];
          if (pe >= cap_e || pi >= cap_i) {
            atomicCAS(&ctrl->error, 0, kErrCapacity);
          } else {
            born_pair<R, false>(P, me, mi, pe, pi, me.cell[o], me.off[o], me.wj[o], me.id[o],
                                step, es[u], se.next_id + rank, si.next_id + rank);
          }
        }
        before += (uint32_t)(rows >> (16 * u)) & 0xFFFFu;
      }
      // electrons emitted at the cathode, after every ionization electron
      const uint32_t n_ionz = before;
      const SoAT<R> sb = soa_as<R>(E.stage_b);
      for (uint32_t e = t; e < sh.tot[1]; e += kSmallThreads) {
        const int j = tile_of_event(sh.pre[1], (int)si.n_tiles, e);
        const size_t o = (size_t)j * kTile + (e - sh.pre[1][j]);
        const uint32_t rank = n_ionz + e;
        const uint32_t pe = app_e + rank;
        if (pe >= cap_e) {
          atomicCAS(&ctrl->error, 0, kErrCapacity);
          continue;
        }
        me.cell[pe] = sb.cell[o];
        me.off[pe] = sb.off[o];
        me.vx[pe] = sb.vx[o];
        me.vy[pe] = sb.vy[o];
        me.vz[pe] = sb.vz[o];
        me.wj[pe] = sb.wj[o];
        me.id[pe] = kGenBit | ((se.next_id + rank) & kSerialMask);
      }
    }
    __syncthreads();
    if (*((volatile int*)&ctrl->error)) break;  // the step is not committed

    // ---- 3. counts, fills and where the stores end ---------------------------
    if (t < 2) {
      const int sp = t;
      const uint32_t n_ionz = (uint32_t)sh.acc[ACC_COLL2], n_see = (uint32_t)sh.acc[ACC_SEE];
      const uint32_t absorbed =
          (uint32_t)(sh.acc[ACC_NABS + 2 * sp] + sh.acc[ACC_NABS + 2 * sp + 1]);
      const uint32_t nb = sp ? n_ionz : n_ionz + n_see;
      const SpeciesState s0 = sh.st[sp];
      const uint32_t tail =
          s0.n_tiles ? (s0.n_tiles - 1) * (uint32_t)kTile + sh.fill[sp][s0.n_tiles - 1] : 0u;
      const uint32_t end = tail + nb;
      const uint32_t n_new = s0.n_live - absorbed + nb;
      const uint32_t nt = (end + kTile - 1) / kTile;
      sh.tail[sp] = tail;
      sh.end[sp] = end;
      sh.n_new[sp] = n_new;
      sh.nt[sp] = nt;
      sh.nb[sp] = nb;
      // repack when under three quarters of the slots in use are live
      sh.compact[sp] =
          (nt > 2 && (unsigned long long)n_new * 4 < (unsigned long long)nt * kTile * 3) ? 1u : 0u;
    }
    __syncthreads();
    for (int sp = 0; sp < 2; ++sp) {
      if (sh.end[sp] == sh.tail[sp]) continue;
      for (uint32_t k = sh.tail[sp] / kTile + t; k < sh.nt[sp]; k += kSmallThreads)
        sh.fill[sp][k] = min(sh.end[sp] - k * (uint32_t)kTile, (uint32_t)kTile);
    }
    __syncthreads();
    // ---- repacking of a sparse store into its other buffer, in order --------
    for (int sp = 0; sp < 2; ++sp) {
      if (!sh.compact[sp]) continue;
      if (warp == 0) warp_prefix(sh.fill[sp], (int)sh.nt[sp], sh.pre[sp]);
      __syncthreads();
      const SpeciesDev& S = P.sp[sp];
      const SoAT<R> src = soa_as<R>(S.buf[sh.st[sp].cur]), dst = soa_as<R>(S.buf[sh.st[sp].cur ^ 1u]);
      for (uint32_t k = warp; k < sh.nt[sp]; k += kSmallWarps) {
        const uint32_t n = sh.fill[sp][k];
        const size_t from = (size_t)k * kTile, to = sh.pre[sp][k];
        for (uint32_t i = lane; i < n; i += 32) {
          dst.cell[to + i] = src.cell[from + i];
          dst.off[to + i] = src.off[from + i];
          dst.vx[to + i] = src.vx[from + i];
          dst.vy[to + i] = src.vy[from + i];
          dst.vz[to + i] = src.vz[from + i];
          dst.wj[to + i] = src.wj[from + i];
          dst.id[to + i] = src.id[from + i];
        }
      }
      __syncthreads();
      const uint32_t nt_new = (sh.n_new[sp] + kTile - 1) / kTile;
      for (uint32_t k = t; k < nt_new; k += kSmallThreads)
        sh.fill[sp][k] = min(sh.n_new[sp] - k * (uint32_t)kTile, (uint32_t)kTile);
      __syncthreads();
    }
    if (t < 2) {
      SpeciesState& s = sh.st[t];
      if (sh.compact[t]) s.cur ^= 1u;
      s.n_tiles = sh.compact[t] ? (sh.n_new[t] + kTile - 1) / kTile : sh.nt[t];
      s.n_live = sh.n_new[t];
      s.next_id += sh.nb[t];
    }
    __syncthreads();

    // ---- deposit and field (field mode 1) ------------------------------------
    if (poisson) {
      deposit_all<R>(P, sh, s_rho0, s_rho1);
      __syncthreads();
      long long* s_net = reinterpret_cast<long long*>(s_rho0);
      for (int k = t; k < nn; k += kSmallThreads) {
        s_net[k] = (long long)s_rho1[k] - (long long)s_rho0[k];
        s_rho1[k] = 0ull;
      }
      __syncthreads();
      // E_k = -(2 D_1 - C (I_k + I_{k+1})) / (2 dx), one-sided at the
      // electrodes, with the exact integer sums of the batched finish kernel
      const int chunk = (N + kSmallThreads - 1) / kSmallThreads;  // over k = 1..N
      const int k0 = 1 + t * chunk;
      long long I0;
      const double D1 = poisson_d1<kSmallThreads>(P, s_net, k0, chunk, sh.i64, sh.i128, &I0);
      const double C = P.pois_C;
      const double inv2dx = 1.0 / (2.0 * P.dx);
      const double twoD1 = D1 + D1;
      long long Ik = I0;
      for (int k = k0; k < k0 + chunk && k <= N; ++k) {
        double e;
        if (k <= N - 1) {
          const long long Ik1 = Ik + s_net[k];
          e = -(twoD1 - C * (double)(Ik + Ik1)) * inv2dx;
          Ik = Ik1;
        } else {
          e = -(D1 - C * (double)Ik) / P.dx;  // k = N
        }
        s_E[k] = e;
      }
      if (t == 0) s_E[0] = -D1 / P.dx;
      __syncthreads();
      for (int k = t; k < nn; k += kSmallThreads) s_rho0[k] = 0ull;
    }

    // ---- tallies ---------------------------------------------------------------
    if (t < kTallySlots)
      commit_tally_slot(P, t, sh.acc, sh.step, sh.n_steps_done, sh.st[0].n_live,
                        sh.st[1].n_live, sh.w_live, &sh.ion_steps);
    __syncthreads();
    if (t < ACC_COUNT) sh.acc[t] = 0ull;
    if (t == 0) {
      sh.step += 1u;
      sh.n_steps_done += 1;
    }
    ++done;
  }

  // ---- the state back to global memory ------------------------------------------
  __syncthreads();
  if (t < 2) r.sstate[inst * 2 + t] = sh.st[t];
  if (t == 0) {
    gis.step = sh.step;
    gis.n_steps_done = sh.n_steps_done;
    gis.w_live[0] = sh.w_live[0];
    gis.w_live[1] = sh.w_live[1];
    gis.ion_steps = sh.ion_steps;
    if (inst == 0) ctrl->small_done = done;
  }
  for (int sp = 0; sp < 2; ++sp) {
    const uint32_t n = min(sh.st[sp].n_tiles, (uint32_t)kSmallFillCap);
    for (uint32_t k = t; k < n; k += kSmallThreads) P.sp[sp].fill[sh.st[sp].cur][k] = sh.fill[sp][k];
  }
  if (done == 0) return;
  if (poisson) {
    for (int k = t; k < nn; k += kSmallThreads) {
      P.E64[k] = s_E[k];
      P.E32[k] = (float)s_E[k];
    }
  }
  // the last step's deposit (with an imposed field it is formed when read)
  if (!poisson) return;
  for (int k = t; k < nn; k += kSmallThreads) {
    P.rho_last[kElectron][k] = 0;
    P.rho_last[kIon][k] = 0;
  }
  __syncthreads();
  deposit_all<R>(P, sh, reinterpret_cast<unsigned long long*>(P.rho_last[kElectron]),
                 reinterpret_cast<unsigned long long*>(P.rho_last[kIon]));
}

// Dynamic shared memory of k_small for the largest field-mode-1 grid of
// max_poisson_nodes nodes (0: none), and the resident CTAs per SM.
int small_config(int fp64, int max_poisson_nodes, size_t* smem_bytes, int* blocks_per_sm) {
  const size_t bytes = (size_t)max_poisson_nodes * 24;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return (int)e;
  const void* fn = fp64 ? (const void*)k_small<double> : (const void*)k_small<float>;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return (int)e;
  if (bytes + fa.sharedSizeBytes > (size_t)optin) {
    *smem_bytes = bytes;
    *blocks_per_sm = 0;
    return 0;
  }
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return (int)e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kSmallThreads, bytes);
  *smem_bytes = bytes;
  return (int)e;
}

int launch_small(const DeviceRefs& r, long long n_steps, int max_tiles, size_t smem_bytes,
                 cudaStream_t s) {
  const void* fn = r.fp64 ? (const void*)k_small<double> : (const void*)k_small<float>;
  DeviceRefs rr = r;
  void* args[] = {&rr, &n_steps, &max_tiles};
  if (r.n_inst == 1)
    return (int)cudaLaunchKernel(fn, dim3(1), dim3(kSmallThreads), args, smem_bytes, s);
  return (int)cudaLaunchCooperativeKernel(fn, dim3(r.n_inst), dim3(kSmallThreads), args,
                                          smem_bytes, s);
}

}  // namespace slpic
