// The particle kernel of one SLPIC-MCC step, batched over instances and
// species: gather, speed-limited kick and drift (Eqs. slpicEOMx, slpicEOMv,
// betaAbrupt), absorbing electrodes with ion-induced secondary emission
// (Sec. IV), the null-collision test of electrons against the majorant
// probability (Sec. III; one Philox2x32-10 draw keyed by (id, step)),
// in-place compaction of survivors, and the
// fixed-point deposit of w_p = beta w_j (Eq. Ansatz).
//
// Work decomposition.  Every (instance, species) segment is a sequence of
// tiles of kTile marker slots (tile k holds fill[k] markers).  A persistent
// grid takes the tiles round-robin (CTA c: tiles c, c + G, c + 2G, ...);
// tiles are independent, so no CTA ever waits for another.  Per CTA the tiles
// go through a two-stage shared-memory pipeline:
//   - bulk asynchronous copies (TMA, cp.async.bulk) bring the seven SoA
//     streams of the next tile into one stage while the current tile is
//     advanced in the other;
//   - each thread advances the markers of slots t and t + kThreads in place
//     in the stage and deposits the survivors into a shared-memory copy of the
//     segment's charge grid (integer atomics);
//   - warp ballots and one scan over the warps rank survivors and events
//     (ion emissions, electron collision candidates); when a marker left the
//     tile the survivors are compacted in order; the fields that changed are
//     stored to the tile's own slots with bulk copies.
// Collision candidates (the electrons that drew u < P0) are not scattered
// here: their final slots are queued per tile and k_collide scatters them
// all at once, so the long, rare scattering path never stalls the stream.
// The shared charge grid is added to global memory with integer atomics when
// the CTA moves to another segment or finishes, so the deposit is exact and
// independent of the order of the additions.
#include "device_common.cuh"
#include "slpic_internal.h"

namespace slpic {

namespace {

constexpr int kWarps = kThreads / 32;

struct TileInfo {
  unsigned int g;     // global tile index (>= n_tiles: none)
  int seg;            // segment = instance * 2 + species
  unsigned int k;     // tile inside the segment
  unsigned int fill;  // live markers in the tile
};

struct CtaShared {
  unsigned long long warp_cnt[kWarps];  // packed counts per warp (16-bit fields)
  unsigned long long warp_pre[kWarps];  // their exclusive prefix over warps
  unsigned long long tot;               // their totals
  unsigned long long s_acc[ACC_COUNT];
  uint64_t bar[2];
  TileInfo cur;
  int abort;
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

// Segment and tile of global tile g (g < n_tiles) and its fill.
__device__ __forceinline__ TileInfo locate(const DeviceRefs& r, unsigned int n_tiles,
                                           unsigned int g) {
  TileInfo t;
  t.g = g;
  t.seg = -1;
  t.k = 0;
  t.fill = 0;
  if (g < n_tiles) {
    int lo = 0, hi = r.n_inst * 2 - 1;  // last segment with seg_start <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (r.seg_start[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    t.seg = lo;
    t.k = g - r.seg_start[lo];
    t.fill = r.inst[lo >> 1].sp[lo & 1].fill[r.sstate[lo].cur][t.k];
  }
  return t;
}

// Start the bulk loads of tile t into `stage` (thread 0).
__device__ __forceinline__ void load_tile(const DeviceRefs& r, const TileInfo& t, float* stage,
                                          uint64_t* bar) {
  if (t.seg < 0 || t.fill == 0) return;
  const SpeciesDev& S = r.inst[t.seg >> 1].sp[t.seg & 1];
  const SoA in = S.buf[r.sstate[t.seg].cur];
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

// A marker left the gap: tally the flux through the electrode (Eq. j); an ion
// at the cathode emits an electron with probability gamma.  Returns true when
// an electron is emitted.  Rare; kept out of line.
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
  // static schedule: this CTA takes tiles blockIdx.x + n gridDim.x; thread 0
  // keeps the next two in registers so that their fills are loaded a whole
  // tile ahead of their bulk loads
  TileInfo nxt, nxt2;
  if (threadIdx.x == 0) {
    mbar_init(&cs.bar[0], 1);
    mbar_init(&cs.bar[1], 1);
    fence_mbar_init();
    cs.abort = 0;
    const TileInfo first = locate(r, n_tiles, blockIdx.x);
    load_tile(r, first, stage0, &cs.bar[0]);
    cs.cur = first;
    nxt = locate(r, n_tiles, blockIdx.x + gridDim.x);
    nxt2 = locate(r, n_tiles, blockIdx.x + 2 * gridDim.x);
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
      load_tile(r, nxt, stage_idx ? stage0 : stage1, &cs.bar[stage_idx ^ 1]);
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
    const float qmdt = S.qmdt, vlim = S.vlim, dtdx = P.dtdx, P0 = P.P0;
    const int N = P.n_cells, shift = P.charge_shift;
    const float* E32 = P.E32;
    const uint32_t key2 = P.key2;
    const bool electrons = sp == kElectron;

    // ---- 1. advance the thread's slots in place ------------------------------
    // event: an ion emitting an electron at the cathode, or an electron that
    // is a null-collision candidate
    uint32_t alive_bits = 0, event_bits = 0;
    uint32_t b_alive[kPerThread], b_event[kPerThread];
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
      const int i = j * kThreads + threadIdx.x;
      bool alive = false, event = false;
      if (i < (int)t.fill && !cs.abort) {
        int cell = st_cell[i];
        float off = st_off[i], vx = st_vx[i];
        const float vy = st_vy[i], vz = st_vz[i];
        // gather (linear between the cell's nodes)
        const float E0 = __ldg(E32 + cell), E1 = __ldg(E32 + cell + 1);
        const float Ex = E0 + off * (E1 - E0);
        // speed-limited kick (beta of the pre-kick speed) and drift (beta of
        // the post-kick speed)
        const float s0 = vx * vx + vy * vy + vz * vz;
        const float b0 = beta_of(sqrtf(s0), vlim);
        vx = vx + b0 * (qmdt * Ex);
        const float s1 = vx * vx + vy * vy + vz * vz;
        const float b1 = beta_of(sqrtf(s1), vlim);
        off = off + b1 * (vx * dtdx);
        const float fl = floorf(off);
        cell += (int)fl;
        off = off - fl;
        if (off >= 1.0f) {
          off = 0.0f;
          cell += 1;
        }
        if (cell < 0 || cell >= N) {
          event = absorb(P, sp, cell < 0 ? 0 : 1, st_wj[i], st_id[i], step, cs.s_acc);
        } else {
          alive = true;
          if (electrons) {
            const uint2 rr = philox2x32_10(make_uint2(st_id[i], step), key2);
            event = uniform01(rr.x) < P0;
          }
          // deposit w_p = beta w_j now unless a collision may change v
          if (!event) deposit(rho, cell, off, fixed_charge(b1 * st_wj[i], shift));
          st_cell[i] = cell;
          st_off[i] = off;
          st_vx[i] = vx;
        }
      }
      b_alive[j] = __ballot_sync(0xFFFFFFFFu, alive);
      b_event[j] = __ballot_sync(0xFFFFFFFFu, event);
      alive_bits |= (alive ? 1u : 0u) << j;
      event_bits |= (event ? 1u : 0u) << j;
    }

    // ---- 2. rank survivors and events inside the tile ------------------------
    // packed word: alive pass 0 | alive pass 1 | events pass 0 | events pass 1
    if (lane == 0) {
      cs.warp_cnt[warp] = (unsigned long long)__popc(b_alive[0]) |
                          ((unsigned long long)__popc(b_alive[1]) << 16) |
                          ((unsigned long long)__popc(b_event[0]) << 32) |
                          ((unsigned long long)__popc(b_event[1]) << 48);
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
    const uint32_t n_event = field16(tot, 2) + field16(tot, 3);
    const size_t tbase = (size_t)t.k * kTile;

    // ---- 3. events: emissions to staging, candidates to the queue -------------
    if (event_bits) {
#pragma unroll
      for (int j = 0; j < kPerThread; ++j) {
        if (!(event_bits >> j & 1u)) continue;
        const int i = j * kThreads + threadIdx.x;
        const uint32_t e = (j ? field16(tot, 2) : 0u) + field16(pre, 2 + j) +
                           (uint32_t)__popc(b_event[j] & lanemask_lt);
        if (electrons) {
          // the candidate's slot after compaction = its rank among survivors
          const uint32_t a = (j ? field16(tot, 0) : 0u) + field16(pre, j) +
                             (uint32_t)__popc(b_alive[j] & lanemask_lt);
          S.cand[tbase + e] = (uint16_t)a;
        } else {
          stage_emission(P, tbase + e, st_wj[i]);
        }
      }
    }

    // ---- 4. compact the survivors in place (only if a marker left) ----------
    const bool compact = n_surv != t.fill;
    if (compact) {
      int32_t c_cell[kPerThread];
      float c_off[kPerThread], c_vx[kPerThread], c_vy[kPerThread], c_vz[kPerThread],
          c_wj[kPerThread];
      uint32_t c_id[kPerThread];
#pragma unroll
      for (int j = 0; j < kPerThread; ++j) {
        const int i = j * kThreads + threadIdx.x;
        if (alive_bits >> j & 1u) {
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
    }
    fence_proxy_async_smem();
    __syncthreads();

    // ---- 5. store the tile to its own slots -----------------------------------
    // position and vx change every step; vy, vz, w_j and the id only move here
    // when the tile was compacted (collisions write vy, vz in k_collide)
    if (threadIdx.x == 0) {
      if (n_surv) {
        const SoA out = S.buf[r.sstate[t.seg].cur];
        const uint32_t bytes = ((n_surv + 3u) & ~3u) * 4u;
        bulk_store(out.cell + tbase, st + 0 * kTile, bytes);
        bulk_store(out.off + tbase, st + 1 * kTile, bytes);
        bulk_store(out.vx + tbase, st + 2 * kTile, bytes);
        if (compact) {
          bulk_store(out.vy + tbase, st + 3 * kTile, bytes);
          bulk_store(out.vz + tbase, st + 4 * kTile, bytes);
          bulk_store(out.wj + tbase, st + 5 * kTile, bytes);
          bulk_store(out.id + tbase, st + 6 * kTile, bytes);
        }
        bulk_commit();
      }
      S.fill[r.sstate[t.seg].cur][t.k] = n_surv;
      if (electrons) S.n_cand[t.k] = n_event;
      else S.births[t.k] = n_event;
      atomicAdd(&cs.s_acc[ACC_MSTEPS], (unsigned long long)t.fill);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      cs.cur = nxt;
      nxt = nxt2;
      nxt2 = locate(r, n_tiles, nxt.g + gridDim.x);
    }
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
