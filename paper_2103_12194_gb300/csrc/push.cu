// The particle kernel of one SLPIC-MCC step, batched over instances and
// species: gather, speed-limited kick and drift (Eqs. slpicEOMx, slpicEOMv,
// betaAbrupt), absorbing electrodes with ion-induced secondary emission
// (Sec. IV), the null-collision test of electrons against the majorant
// probability (Sec. III; one Philox2x32-10 draw keyed by (id, step)),
// in-place compaction of survivors, and the fixed-point deposit of
// w_p = beta w_j (Eq. Ansatz; with an imposed field the deposit is formed
// from the markers when read, and the step deposits nothing).
//
// Work decomposition.  Every (instance, species) segment is a sequence of
// tiles of kTile = 128 marker slots (tile k holds fill[k] markers), and every
// tile belongs to one warp: no block-wide barrier is needed to advance,
// rank, compact and store it.
//   - A CTA of W warps takes super-tiles of W consecutive tiles of one
//     segment (warp w: tile w of each); the CTAs split the super-tiles into
//     contiguous ranges of equal weight, so a CTA deposits into few segments.
//   - Each warp streams its tiles through three shared-memory stages: lane 0
//     starts the bulk asynchronous copies (TMA, cp.async.bulk) of the seven
//     SoA streams of the tile two rounds ahead while the warp advances the
//     current one, so two tiles per warp are in flight.
//   - Lane l advances slots l, l + 32, l + 64, l + 96 (read into registers)
//     and deposits the survivors into a shared-memory copy of the segment's
//     charge grid (integer atomics).
//   - Ballots rank survivors and events (ion emissions, electron collision
//     candidates); the survivors go back to the stage, compacted in order
//     when a marker left the tile, and lane 0 stores the fields that changed
//     to the tile's own slots with bulk copies.
// Collision candidates (the electrons that drew u < P0) are not scattered
// here: their states and final slots are queued per tile as 32-byte records
// and k_collide scatters them all at once, so the long, rare scattering path
// never stalls the stream and reads each candidate with one sector.
// The shared charge grid is added to global memory with integer atomics when
// the CTA moves to another segment (a CTA-wide barrier, taken by all warps at
// the same round) or finishes, so the deposit is exact and independent of the
// order of the additions.
#include "device_common.cuh"
#include "slpic_internal.h"
#include "step_ops.cuh"

namespace slpic {

namespace {

// Tile of a warp in one round: the super-tile's segment (CTA-uniform) and,
// when the warp has a tile there, its index and fill.
struct WarpTile {
  int sseg;       // segment of the super-tile
  bool valid;     // the warp has a tile in it
  uint32_t k;     // tile inside the segment
  uint32_t fill;  // live markers in the tile
};

struct PushShared {
  unsigned long long s_acc[ACC_COUNT];
  int abort;
};

__device__ __forceinline__ void set_error(Control* ctrl, int code) {
  atomicCAS(&ctrl->error, 0, code);
}

// Add the CTA's shared charge grid and accumulators of segment seg to global
// memory and clear them (all threads; barriers before and after).
__device__ __forceinline__ void flush_segment(const DeviceRefs& r, int seg,
                                              unsigned long long* s_rho, PushShared& cs,
                                              bool use_smem) {
  const int inst = seg >> 1, sp = seg & 1;
  const InstDev& P = r.inst[inst];
  __syncthreads();
  if (use_smem) {
    const int nn = P.n_cells + 1;
    unsigned long long* g = P.rho_acc[sp];
    for (int k = threadIdx.x; k < nn; k += blockDim.x) {
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

// Segment of super-tile q (q < n_super): the last segment starting at or
// before q.
__device__ __forceinline__ int segment_of(const DeviceRefs& r, unsigned int q) {
  int lo = 0, hi = r.n_inst * 2 - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (r.seg_start[mid] <= q) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// First super-tile whose weighted start is at or after `target`.
__device__ __forceinline__ unsigned int first_super(const DeviceRefs& r, unsigned int target) {
  const int n_seg = r.n_inst * 2;
  if (target >= r.seg_wstart[n_seg]) return r.seg_start[n_seg];
  int lo = 0, hi = n_seg - 1;  // last segment with weighted start <= target
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (r.seg_wstart[mid] <= target) lo = mid;
    else hi = mid - 1;
  }
  const unsigned int w = (lo & 1) ? kWeightIon : kWeightElectron;
  const unsigned int q = r.seg_start[lo] + (target - r.seg_wstart[lo] + w - 1) / w;
  return min(q, r.seg_start[lo + 1]);
}

// A warp's look-ahead stays in one segment for many rounds: the segment of
// the last super-tile looked up, with its super-tile range, tile count and
// fill array, so that a round costs one load (the fill) instead of a search
// and a chain of dependent loads.
struct SegCursor {
  int seg;
  unsigned int q_begin, q_end;  // super-tiles of the segment
  uint32_t n_tiles;
  const uint32_t* fill;
};

__device__ __forceinline__ WarpTile tile_of(const DeviceRefs& r, SegCursor& c, unsigned int q,
                                            int warp) {
  if (q < c.q_begin || q >= c.q_end) {
    c.seg = segment_of(r, q);
    c.q_begin = r.seg_start[c.seg];
    c.q_end = r.seg_start[c.seg + 1];
    const SpeciesState& st = r.sstate[c.seg];
    c.n_tiles = st.n_tiles;
    c.fill = r.inst[c.seg >> 1].sp[c.seg & 1].fill[st.cur];
  }
  WarpTile t;
  t.sseg = c.seg;
  t.k = (q - c.q_begin) * (uint32_t)r.push_warps + (uint32_t)warp;
  t.valid = t.k < c.n_tiles;
  t.fill = t.valid ? c.fill[t.k] : 0u;
  return t;
}

// Views of a tile's stage: cell and id, then the five real streams.
template <typename R>
struct Stage {
  int32_t* cell;
  uint32_t* id;
  R* f[5];  // off, vx, vy, vz, w_j
  __device__ __forceinline__ explicit Stage(unsigned char* base) {
    cell = reinterpret_cast<int32_t*>(base);
    id = reinterpret_cast<uint32_t*>(base + kTile * 4);
    R* rr = reinterpret_cast<R*>(base + kTile * 8);
#pragma unroll
    for (int q = 0; q < 5; ++q) f[q] = rr + q * kTile;
  }
};

// Start the bulk loads of tile t into `stage` (lane 0).
template <typename R>
__device__ __forceinline__ void load_tile(const DeviceRefs& r, const WarpTile& t,
                                          unsigned char* stage, uint64_t* bar) {
  const SpeciesDev& S = r.inst[t.sseg >> 1].sp[t.sseg & 1];
  const SoAT<R> in = soa_as<R>(S.buf[r.sstate[t.sseg].cur]);
  const size_t base = (size_t)t.k * kTile;
  const uint32_t n4 = (t.fill + 3u) & ~3u;  // 16-byte multiples
  const uint32_t b4 = n4 * 4u, br = n4 * (uint32_t)sizeof(R);
  Stage<R> st(stage);
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(bar, 2u * b4 + 5u * br);
  bulk_load(st.cell, in.cell + base, b4, bar);
  bulk_load(st.id, in.id + base, b4, bar);
  bulk_load(st.f[0], in.off + base, br, bar);
  bulk_load(st.f[1], in.vx + base, br, bar);
  bulk_load(st.f[2], in.vy + base, br, bar);
  bulk_load(st.f[3], in.vz + base, br, bar);
  bulk_load(st.f[4], in.wj + base, br, bar);
}

}  // namespace

template <typename R>
__global__ void __launch_bounds__(kPushMaxWarps * 32, 1) k_push(DeviceRefs r) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t s_bar[kPushMaxWarps][kPushStages];
  __shared__ PushShared cs;
  const int W = (int)(blockDim.x >> 5);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lanemask_lt = (1u << lane) - 1u;
  constexpr int kSB = stage_bytes<R>();
  unsigned char* stages = smem_raw + (size_t)warp * kPushStages * kSB;
  unsigned long long* s_rho =
      reinterpret_cast<unsigned long long*>(smem_raw + (size_t)W * kPushStages * kSB);
  uint64_t* bars = s_bar[warp];

  step_kernel_entry();
  Control* ctrl = r.ctrl;
  if (*((volatile int*)&ctrl->error)) return;
  const uint32_t limit = spin_limit(ctrl);
  // this CTA's contiguous range of super-tiles (equal weight per CTA)
  const unsigned long long wt = ctrl->w_total;
  const unsigned int q0 =
      first_super(r, (unsigned int)((unsigned long long)blockIdx.x * wt / gridDim.x));
  const unsigned int q1 =
      first_super(r, (unsigned int)((unsigned long long)(blockIdx.x + 1) * wt / gridDim.x));
  const int n_rounds = (int)(q1 - q0);

  for (int k = threadIdx.x; k < r.smem_nodes; k += blockDim.x) s_rho[k] = 0ull;
  if (threadIdx.x < ACC_COUNT) cs.s_acc[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) cs.abort = 0;
  if (lane == 0) {
    for (int s = 0; s < kPushStages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  volatile int* abort_flag = &cs.abort;

  SegCursor cursor;
  cursor.seg = 0;
  cursor.q_begin = 1u;  // empty range: the first look-up searches
  cursor.q_end = 0u;
  cursor.n_tiles = 0u;
  cursor.fill = nullptr;
  // descriptors of rounds m .. m + kPushStages (the bulk loads of a round
  // are issued kPushStages - 1 rounds ahead, and its fill is read a round
  // before that)
  constexpr int kAhead = kPushStages - 1;
  WarpTile d[kPushStages + 1];
#pragma unroll
  for (int j = 0; j <= kPushStages; ++j) {
    d[j].valid = false;
    d[j].fill = 0u;
    d[j].sseg = 0;
    d[j].k = 0u;
  }
#pragma unroll
  for (int j = 0; j < kPushStages; ++j)
    if (j < n_rounds) d[j] = tile_of(r, cursor, q0 + j, warp);
  uint32_t phase = 0;    // parity bit per stage
  uint32_t pending = 0;  // stages with a bulk load not yet waited for
#pragma unroll
  for (int j = 0; j < kAhead; ++j) {
    if (d[j].valid && d[j].fill) {
      if (lane == 0) load_tile<R>(r, d[j], stages + j * kSB, &bars[j]);
      pending |= 1u << j;
    }
  }

  int cur_seg = -1;
  bool use_smem = false;
  for (int m = 0; m < n_rounds; ++m) {
    // ---- 0. descriptors ahead; bulk loads of round m + kAhead ---------------
    if (m + kPushStages < n_rounds) d[kPushStages] = tile_of(r, cursor, q0 + m + kPushStages, warp);
    const int sc = m % kPushStages;             // stage of round m
    const int sn = (m + kAhead) % kPushStages;  // stage of round m + kAhead
    const bool aborted = *abort_flag != 0;
    if (m + kAhead < n_rounds && d[kAhead].valid && d[kAhead].fill && !aborted) {
      if (lane == 0) {
        // the stage's last bulk stores (round m - 1) must have read it
        bulk_wait_read_all();
        load_tile<R>(r, d[kAhead], stages + sn * kSB, &bars[sn]);
      }
      pending |= 1u << sn;
    }
    // ---- 1. segment change: flush the shared grid (all warps, same round) ----
    if (d[0].sseg != cur_seg) {
      if (cur_seg >= 0) flush_segment(r, cur_seg, s_rho, cs, use_smem);
      cur_seg = d[0].sseg;
      // with an imposed field the deposit is formed from the markers when it
      // is read (k_deposit), so nothing is deposited here
      use_smem = r.inst[cur_seg >> 1].field_mode == 1 &&
                 r.inst[cur_seg >> 1].n_cells + 1 <= r.smem_nodes;
    }

    const WarpTile t = d[0];
    if (t.valid && !aborted) {
      const int inst = t.sseg >> 1, sp = t.sseg & 1;
      const InstDev& P = r.inst[inst];
      const SpeciesDev& S = P.sp[sp];
      const uint32_t cur_buf = r.sstate[t.sseg].cur;
      const size_t tbase = (size_t)t.k * kTile;
      uint32_t n_surv = 0, n_event = 0;
      bool compact = false;
      const Stage<R> st(stages + sc * kSB);
      int32_t* st_cell = st.cell;
      R* st_off = st.f[0];
      R* st_vx = st.f[1];
      R* st_vy = st.f[2];
      R* st_vz = st.f[3];
      R* st_wj = st.f[4];
      uint32_t* st_id = st.id;
      // ---- 2. the tile's data: wait (bounded), then read it into registers -----
      bool ok = true;
      if (t.fill) {
        uint32_t polls = 0;
        while (!mbar_try_wait(&bars[sc], (phase >> sc) & 1u)) {
          if (++polls > limit) {
            set_error(ctrl, kErrTimeout);
            *abort_flag = 1;
            ok = false;
            break;
          }
        }
        ok = __all_sync(0xFFFFFFFFu, ok);
        if (ok) {
          phase ^= 1u << sc;
          pending &= ~(1u << sc);
        }
        if (lane == 0 && polls) {
          atomicAdd(&ctrl->spin_waits, 1u);
          atomicMax(&ctrl->spin_max, polls);
        }
      }
      if (t.fill && ok) {
        unsigned long long* rho = use_smem ? s_rho : P.rho_acc[sp];
        const uint32_t step = r.istate[inst].step;
        const StepConsts<R>& K = consts<R>(P);
        const R qmdt = K.qmdt[sp], vlim = K.vlim[sp], dtdx = K.dtdx, P0 = K.P0;
        const R wscale = K.wscale;
        const uint32_t N = (uint32_t)P.n_cells;
        const R* Enode = node_field<R>(P);
        const bool electrons = sp == kElectron;
        const bool limited = vlim < (R)INFINITY;  // beta = 1 for an unlimited species
        const bool dep = P.field_mode == 1;       // deposit during the step
        // The lane's slots are advanced in kHalves passes of kPerHalf slots
        // (lane l, pass h: slots (h kPerHalf + j) 32 + l), so that one pass's
        // state fits the registers of a CTA of kPushMaxWarps warps.  Ranks of
        // survivors and events run on across the passes, in slot order.
#pragma unroll 1
        for (int h = 0; h < kHalves; ++h) {
          const int i0 = h * kPerHalf * 32;
          if (i0 >= (int)t.fill) break;
          // slots past the fill are read (stage memory) but never used; their
          // cell is taken as 0 so that the gather stays in range
          int cell[kPerHalf];
          R off[kPerHalf], vx[kPerHalf], vy[kPerHalf], vz[kPerHalf], wj[kPerHalf];
          uint32_t id[kPerHalf];
          bool live[kPerHalf];
#pragma unroll
          for (int j = 0; j < kPerHalf; ++j) {
            const int i = i0 + j * 32 + lane;
            live[j] = i < (int)t.fill;
            cell[j] = live[j] ? st_cell[i] : 0;
            off[j] = st_off[i];
            vx[j] = st_vx[i];
            vy[j] = st_vy[i];
            vz[j] = st_vz[i];
            wj[j] = st_wj[i];
            id[j] = st_id[i];
          }
          // ---- 4. advance the slots -------------------------------------------
          R a[kPerHalf], b1[kPerHalf];
#pragma unroll
          for (int j = 0; j < kPerHalf; ++j) {
            // gather (linear between the cell's nodes)
            const R E0 = __ldg(Enode + cell[j]), E1 = __ldg(Enode + cell[j] + 1);
            a[j] = qmdt * (E0 + off[j] * (E1 - E0));
          }
          // speed-limited kick (limited_kick_n: leapfrog below the limit, the
          // exact solution of Eq. slpicEOMv across and above it) and drift
          // (beta of the post-kick speed); an unlimited species has beta = 1
          if (limited) {
#pragma unroll
            for (int j = 0; j < kPerHalf; ++j) {
              R x1[1] = {vx[j]};
              const R y1[1] = {vy[j]}, z1[1] = {vz[j]}, a1[1] = {a[j]};
              limited_kick_n<R, 1>(x1, y1, z1, a1, vlim);
              vx[j] = x1[0];
            }
#pragma unroll
            for (int j = 0; j < kPerHalf; ++j)
              b1[j] = beta_of(r_sqrt(vx[j] * vx[j] + vy[j] * vy[j] + vz[j] * vz[j]), vlim);
          } else {
#pragma unroll
            for (int j = 0; j < kPerHalf; ++j) {
              vx[j] = vx[j] + a[j];
              b1[j] = (R)1;
            }
          }
#pragma unroll
          for (int j = 0; j < kPerHalf; ++j) {
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
          // ---- 5. electrodes (rare, out of line), candidate draws, deposit -----
          bool alive[kPerHalf], event[kPerHalf];
#pragma unroll
          for (int j = 0; j < kPerHalf; ++j) {
            alive[j] = live[j] && (uint32_t)cell[j] < N;
            event[j] = false;
          }
#pragma unroll
          for (int j = 0; j < kPerHalf; ++j) {
            if (live[j] && !alive[j])
              event[j] = absorb<R>(P, sp, cell[j] < 0 ? 0 : 1, wj[j], id[j], step, cs.s_acc,
                                   vx[j], vy[j], vz[j]);
          }
          if (electrons) {
            const uint32_t key2 = P.key2;
#pragma unroll
            for (int j = 0; j < kPerHalf; ++j) {
              const uint2 rr = philox2x32_10(make_uint2(id[j], step), key2);
              event[j] = alive[j] && uniform01r<R>(rr.x) < P0;
            }
          }
#pragma unroll
          for (int j = 0; j < kPerHalf; ++j) {
            // deposit w_p = beta w_j now unless a collision may change v
            if (dep && alive[j] && !event[j]) {
              const long long Q = fixed_charge(b1[j] * wj[j], wscale);
              const long long right = right_share(Q, off[j]);
              atomicAdd(rho + cell[j], (unsigned long long)(Q - right));
              atomicAdd(rho + cell[j] + 1, (unsigned long long)right);
            }
          }
          // ---- 6. rank survivors and events ----------------------------------
          uint32_t b_alive[kPerHalf], b_event[kPerHalf];
          uint32_t pre_alive[kPerHalf], pre_event[kPerHalf];
#pragma unroll
          for (int j = 0; j < kPerHalf; ++j) {
            b_alive[j] = __ballot_sync(0xFFFFFFFFu, alive[j]);
            b_event[j] = __ballot_sync(0xFFFFFFFFu, event[j]);
            pre_alive[j] = n_surv;
            pre_event[j] = n_event;
            n_surv += __popc(b_alive[j]);
            n_event += __popc(b_event[j]);
          }
          // ---- 7. events: emissions to staging, candidates to the queue --------
#pragma unroll
          for (int j = 0; j < kPerHalf; ++j) {
            if (event[j]) {
              const uint32_t e = pre_event[j] + (uint32_t)__popc(b_event[j] & lanemask_lt);
              if (electrons) {
                // the candidate's slot after compaction = its rank among survivors
                const uint32_t r_a = pre_alive[j] + (uint32_t)__popc(b_alive[j] & lanemask_lt);
                put_cand(S.crec, tbase + e, cell[j], off[j], vx[j], vy[j], vz[j], wj[j], id[j],
                         r_a);
              } else if (dep) {
                stage_emission<R>(P, tbase + e, wj[j]);
              } else {
                stage_emission<R, false>(P, tbase + e, wj[j]);
              }
            }
          }
          // ---- 8. write the pass's survivors back to the stage: in place while
          // no marker of the tile has left, else compacted in order (every lane
          // holds the pass's slots in registers, so one warp barrier separates
          // the reads from the writes; the compacted slots lie below the pass's
          // own, which every lane has read)
          const uint32_t live_so_far = min(t.fill, (uint32_t)(i0 + kPerHalf * 32));
          if (n_surv == live_so_far) {
#pragma unroll
            for (int j = 0; j < kPerHalf; ++j) {
              const int i = i0 + j * 32 + lane;
              if (alive[j]) {
                st_cell[i] = cell[j];
                st_off[i] = off[j];
                st_vx[i] = vx[j];
              }
            }
          } else {
            __syncwarp();
#pragma unroll
            for (int j = 0; j < kPerHalf; ++j) {
              if (alive[j]) {
                const uint32_t r_a = pre_alive[j] + (uint32_t)__popc(b_alive[j] & lanemask_lt);
                st_cell[r_a] = cell[j];
                st_off[r_a] = off[j];
                st_vx[r_a] = vx[j];
                st_vy[r_a] = vy[j];
                st_vz[r_a] = vz[j];
                st_wj[r_a] = wj[j];
                st_id[r_a] = id[j];
              }
            }
          }
          __syncwarp();
        }
        compact = n_surv != t.fill;
      }
      // ---- 9. store the tile to its own slots ---------------------------------
      // position and vx change every step; vy, vz, w_j and the id only move
      // here when the tile was compacted (collisions write vy, vz in k_collide)
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0 && ok) {
        if (n_surv) {
          const SoAT<R> o = soa_as<R>(S.buf[cur_buf]);
          const uint32_t n4 = (n_surv + 3u) & ~3u;  // 16-byte multiples
          const uint32_t b4 = n4 * 4u, br = n4 * (uint32_t)sizeof(R);
          bulk_store(o.cell + tbase, st_cell, b4);
          bulk_store(o.off + tbase, st_off, br);
          bulk_store(o.vx + tbase, st_vx, br);
          if (compact) {
            bulk_store(o.vy + tbase, st_vy, br);
            bulk_store(o.vz + tbase, st_vz, br);
            bulk_store(o.wj + tbase, st_wj, br);
            bulk_store(o.id + tbase, st_id, b4);
          }
          bulk_commit();
        }
        S.fill[cur_buf][t.k] = n_surv;
        if (sp == kElectron) S.n_cand[t.k] = n_event;
        else S.births[t.k] = n_event;
        if (t.fill) atomicAdd(&cs.s_acc[ACC_MSTEPS], (unsigned long long)t.fill);
      }
    }
#pragma unroll
    for (int j = 0; j < kPushStages; ++j) d[j] = d[j + 1];
    d[kPushStages].valid = false;
    d[kPushStages].fill = 0u;
  }
  if (n_rounds > 0) flush_segment(r, cur_seg, s_rho, cs, use_smem);
  if (lane == 0) {
    // no bulk copy may outlive the CTA's shared memory
    bulk_wait_all();
    for (int s = 0; s < kPushStages; ++s) {
      if (!(pending >> s & 1u)) continue;
      const uint32_t ph = (phase >> s) & 1u;
      for (uint32_t p = 0; p < kSpinLimit && !mbar_try_wait(&bars[s], ph); ++p) {
      }
    }
  }
}

template <typename R>
int push_config_t(int smem_nodes, int* warps, int* blocks_per_sm, size_t* smem_bytes) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return (int)e;
  const size_t fixed = sizeof(uint64_t) * kPushMaxWarps * kPushStages + sizeof(PushShared) + 1024;
  *warps = 0;
  *blocks_per_sm = 0;
  // the kernel may use all the dynamic shared memory a CTA can have: every
  // context's launches (of any grid size and shape) stay within that limit,
  // so no context's configuration lowers it under another's
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, k_push<R>);
  if (e != cudaSuccess) return (int)e;
  e = cudaFuncSetAttribute(k_push<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) return (int)e;
  for (int w = kPushMaxWarps; w >= 4; w -= 4) {
    const size_t bytes = (size_t)w * kPushStages * stage_bytes<R>() + (size_t)smem_nodes * 8;
    if (bytes + fixed > (size_t)optin) continue;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_push<R>, w * 32, bytes);
    if (e != cudaSuccess) return (int)e;
    if (bps > 0) {
      *warps = w;
      *blocks_per_sm = bps;
      *smem_bytes = bytes;
      return 0;
    }
  }
  return 0;
}

template <typename R>
int push_bps_t(int warps, int smem_nodes, int* blocks_per_sm) {
  const size_t bytes = (size_t)warps * kPushStages * stage_bytes<R>() + (size_t)smem_nodes * 8;
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_push<R>, warps * 32,
                                                            bytes);
}

int push_blocks_per_sm(int fp64, int warps, int smem_nodes, int* blocks_per_sm) {
  return fp64 ? push_bps_t<double>(warps, smem_nodes, blocks_per_sm)
              : push_bps_t<float>(warps, smem_nodes, blocks_per_sm);
}

int push_config(int fp64, int smem_nodes, int* warps, int* blocks_per_sm, size_t* smem_bytes) {
  return fp64 ? push_config_t<double>(smem_nodes, warps, blocks_per_sm, smem_bytes)
              : push_config_t<float>(smem_nodes, warps, blocks_per_sm, smem_bytes);
}

void launch_push(const DeviceRefs& r, int grid, cudaStream_t s) {
  if (r.fp64) {
    const size_t bytes = (size_t)r.push_warps * kPushStages * stage_bytes<double>() +
                         (size_t)r.smem_nodes * 8;
    launch_step_kernel(k_push<double>, grid, r.push_warps * 32, bytes, s, r);
  } else {
    const size_t bytes = (size_t)r.push_warps * kPushStages * stage_bytes<float>() +
                         (size_t)r.smem_nodes * 8;
    launch_step_kernel(k_push<float>, grid, r.push_warps * 32, bytes, s, r);
  }
}

static_assert(kTile == 32 * kPerLane, "a tile is kPerLane slots per lane of one warp");
static_assert(stage_bytes<float>() % 128 == 0 && stage_bytes<double>() % 128 == 0,
              "stages keep 128-byte alignment");

}  // namespace slpic
