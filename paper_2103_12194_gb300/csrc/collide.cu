// Monte-Carlo collisions of the null-collision candidates queued by the
// particle kernel (Sec. III and IV), and the placement of every birth of the
// step.  For a candidate (an electron that drew u < P0 this step) the process
// is chosen by comparing u' P0 with the cumulative rates
// n_g sigma_k(eps) beta v dt (Eq. SLPICcollisionNumber with beta_n = 1,
// whole-marker collisions); elastic collisions scatter by the Vahedi-Surendra
// angles with the recoil loss, excitation removes its threshold and scatters
// isotropically, ionization shares the excess energy between the primary and
// a born electron and creates an Ar+ at the same position with the same flux
// weight.  Each candidate is then deposited with its new density weight
// (with an imposed field the deposit is formed from the markers when read).
//
// Work: chunks of consecutive tiles handed out in order (electron tiles of an
// instance, then its ion tiles); each warp takes an eighth of a chunk (at
// most 32 tiles).  An instance's electron chunks are sized from its last
// step's candidates per tile (about 256 candidates per warp), so a
// collision-dense instance gets small chunks and many CTAs.  A warp numbers
// the candidates of its tiles in (tile, slot) order and takes them 32 at a
// time, one lane each: it reads each candidate's record (its state and slot,
// one 32-byte sector in float; the next round's records load meanwhile),
// draws the process, deposits null collisions at once and queues the others
// by kind in shared memory, scattered 32 at a time on one code path; only
// the new velocity is written to the candidate's slot.  The births of a
// chunk (ionizations; for ion chunks the electrons the particle kernel
// staged for emission) get their slots from an ordered scan over the chunks
// (decoupled look-back), so they are appended after the last live marker in
// (tile, slot) order -- ionization electrons first, emitted electrons after
// -- with their final serial numbers, whatever the scheduling; they are
// placed 32 at a time.
#include "device_common.cuh"
#include "slpic_internal.h"
#include "step_ops.cuh"

namespace slpic {

namespace {

constexpr int kCollThreads = 256;
constexpr int kQ = 64;  // entries of each queue (a round adds at most 32 to one below 32)

// One warp's collision queues in shared memory (structure of arrays, one
// entry per lane of a drain).  Elastic collisions keep the incident velocity;
// excitations and ionizations (rare; one queue) only the energy.  idx packs
// the candidate's tile in the warp's range (5 bits), its rank among the
// tile's candidates (7 bits) and its slot in the tile (7 bits).
template <typename R>
struct CollQueues {
  uint32_t e_idx[kQ];
  int32_t e_cell[kQ];
  R e_off[kQ], e_wj[kQ], e_vx[kQ], e_vy[kQ], e_vz[kQ], e_eps[kQ], e_u2[kQ], e_u3[kQ];
  uint32_t n_idx[kQ], n_id[kQ], n_k[kQ];
  int32_t n_cell[kQ];
  R n_off[kQ], n_wj[kQ], n_eps[kQ], n_u2[kQ], n_u3[kQ];
};

__host__ __device__ constexpr uint32_t pack_idx(uint32_t j, uint32_t q, uint32_t slot) {
  return j | (q << 5) | (slot << 12);
}

}  // namespace

template <typename R>
__global__ void __launch_bounds__(kCollThreads, 4) k_collide(DeviceRefs r) {
  extern __shared__ __align__(16) unsigned char coll_smem[];
  __shared__ unsigned long long s_acc[ACC_COUNT];
  __shared__ uint32_t s_births[kCollWarps];
  __shared__ uint32_t s_prefix;
  __shared__ unsigned int s_chunk;
  step_kernel_entry();
  Control* ctrl = r.ctrl;
  if (*((volatile int*)&ctrl->error)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lanemask_lt = (1u << lane) - 1u;
  const unsigned int n_chunks = ctrl->n_coll_chunks;
  const unsigned int epoch = ctrl->epoch;
  if (threadIdx.x < ACC_COUNT) s_acc[threadIdx.x] = 0ull;
  int cur_inst = -1;

  for (;;) {
    if (threadIdx.x == 0) s_chunk = atomicAdd(&ctrl->coll_counter, 1u);
    __syncthreads();
    const unsigned int c = s_chunk;
    if (c >= n_chunks) break;
    int inst = 0;
    {
      int lo = 0, hi = r.n_inst - 1;  // last instance with coll_start <= c
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (r.coll_start[mid] <= c) lo = mid;
        else hi = mid - 1;
      }
      inst = lo;
    }
    const InstDev& P = r.inst[inst];
    if (inst != cur_inst) {
      if (cur_inst >= 0 && threadIdx.x < ACC_COUNT && s_acc[threadIdx.x]) {
        atomicAdd(r.inst[cur_inst].acc + threadIdx.x, s_acc[threadIdx.x]);
        s_acc[threadIdx.x] = 0ull;
      }
      cur_inst = inst;
      __syncthreads();
    }
    const SpeciesDev& E = P.sp[kElectron];
    const SpeciesDev& I = P.sp[kIon];
    const SpeciesState& se = r.sstate[inst * 2 + kElectron];
    const SpeciesState& si = r.sstate[inst * 2 + kIon];
    const uint32_t step = r.istate[inst].step;
    const unsigned int first = r.coll_start[inst];
    const unsigned int local = c - first;
    const uint32_t Te = r.coll_tiles[inst];
    const unsigned int e_chunks = (se.n_tiles + Te - 1) / Te;
    const bool ion_chunk = local >= e_chunks;
    const uint32_t nt = ion_chunk ? si.n_tiles : se.n_tiles;
    // this warp's tiles: wt consecutive ones, tile kw + j at lane j
    const uint32_t T = ion_chunk ? (uint32_t)kCollMaxChunkTiles : Te;
    const uint32_t wt = T / kCollWarps;
    const uint32_t kw = (ion_chunk ? local - e_chunks : local) * T + warp * wt;
    const SoAT<R> me = soa_as<R>(E.buf[se.cur]);
    const StepConsts<R>& K = consts<R>(P);
    const R kv = K.K_V[kElectron], vlim = K.vlim[kElectron];
    // events of the tiles (electron chunks: queued candidates; ion chunks:
    // electrons emitted at the cathode) and their exclusive prefix: the
    // warp's events are numbered in (tile, slot) order
    uint32_t cnt = 0;
    if (lane < wt && kw + lane < nt) cnt = ion_chunk ? I.births[kw + lane] : E.n_cand[kw + lane];
    uint32_t excl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t n = __shfl_up_sync(0xFFFFFFFFu, excl, o);
      if (lane >= o) excl += n;
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, excl, 31);
    excl -= cnt;
    // tile (lane index j) and rank inside it of the warp's event number e < total:
    // the last tile whose prefix is <= e (that tile has events)
    auto locate_event = [&](uint32_t e, uint32_t& q) -> int {
      int j = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const uint32_t v = __shfl_sync(0xFFFFFFFFu, excl, j + step);
        if (v <= e) j += step;
      }
      q = e - __shfl_sync(0xFFFFFFFFu, excl, j);
      return j;
    };

    // ---- pass 1: scatter this warp's candidates, count the births ------------
    // Rounds of 32 candidates, one per lane: each lane draws its candidate's
    // process (the records of the next round load meanwhile); null collisions
    // are deposited at once, the others queued by kind and scattered 32 at a
    // time with every lane on the same path.  Each collision's arithmetic is
    // that of collide(); the deposits and counters are integer sums, so the
    // order of the scatterings does not matter.
    uint32_t warp_births = 0;
    if (!ion_chunk && total) {
      CollQueues<R>& Q = reinterpret_cast<CollQueues<R>*>(coll_smem)[warp];
      const uint32_t ctr2 = P.ctr_inst * 2u, key0 = P.key0, key1 = P.key1;
      const bool dep = P.field_mode == 1;  // imposed field: the deposit is formed when read
      unsigned long long* rho_e = P.rho_acc[kElectron];
      const R wscale = K.wscale;
      CandRec<R>* crec = reinterpret_cast<CandRec<R>*>(E.crec);
      const size_t kbase = (size_t)kw * kTile;
      // the new velocity of slot o, and the deposit with it
      auto finish_one = [&](uint32_t o, int cell, R off, R wj, const Velocity<R>& nv) {
        me.vx[o] = nv.vx;
        me.vy[o] = nv.vy;
        me.vz[o] = nv.vz;
        if (dep)
          deposit(rho_e, cell, off,
                  fixed_charge(beta_of(r_sqrt(nv.vx * nv.vx + nv.vy * nv.vy + nv.vz * nv.vz),
                                       vlim) * wj, wscale));
      };
      uint32_t e_head = 0, e_tail = 0, n_head = 0, n_tail = 0;
      // scatter the n <= 32 oldest elastic (inelastic) entries, lane l the l-th
      auto drain_elastic = [&](uint32_t n) {
        const uint32_t i = (e_head + lane) & (kQ - 1);
        const bool on = lane < n;
        uint32_t idx = 0;
        int cell = 0;
        R off = 0, wj = 0, vx = 0, vy = 0, vz = 0, eps = 0, u2 = 0, u3 = 0;
        if (on) {
          idx = Q.e_idx[i];
          cell = Q.e_cell[i];
          off = Q.e_off[i];
          wj = Q.e_wj[i];
          vx = Q.e_vx[i];
          vy = Q.e_vy[i];
          vz = Q.e_vz[i];
          eps = Q.e_eps[i];
          u2 = Q.e_u2[i];
          u3 = Q.e_u3[i];
        }
        __syncwarp();  // the entries are read before the next round refills them
        if (on) {
          const R v1 = r_sqrt(vx * vx + vy * vy + vz * vz);
          const Velocity<R> nv = scatter_elastic<R>(K, kv, vx, vy, vz, v1, eps, u2, u3);
          finish_one((uint32_t)(kbase + (idx & 31u) * kTile + (idx >> 12)), cell, off, wj, nv);
        }
        e_head += n;
      };
      auto drain_inelastic = [&](uint32_t n) {
        const uint32_t i = (n_head + lane) & (kQ - 1);
        const bool on = lane < n;
        uint32_t idx = 0, id = 0, k = 0;
        int cell = 0;
        R off = 0, wj = 0, eps = 0, u2 = 0, u3 = 0;
        if (on) {
          idx = Q.n_idx[i];
          id = Q.n_id[i];
          k = Q.n_k[i];
          cell = Q.n_cell[i];
          off = Q.n_off[i];
          wj = Q.n_wj[i];
          eps = Q.n_eps[i];
          u2 = Q.n_u2[i];
          u3 = Q.n_u3[i];
        }
        __syncwarp();
        if (on) {
          const size_t base = kbase + (idx & 31u) * kTile;
          const uint32_t slot = idx >> 12;
          Velocity<R> nv;
          if ((int)k <= P.n_exc) {
            nv = scatter_excitation<R>(K, kv, eps, (int)k, u2, u3, s_acc);
          } else {
            R es;
            nv = scatter_ionization<R>(P, kv, eps, u2, u3, id, step, wj, s_acc, &es);
            // mark for pass 2, with the secondary's energy in place of vx
            CandRec<R>* w = crec + base + ((idx >> 5) & 127u);
            w->slot = slot | kIonizedMark;
            w->vx = es;
          }
          finish_one((uint32_t)(base + slot), cell, off, wj, nv);
        }
        n_head += n;
      };
      uint32_t qn;
      int jn = locate_event(lane < total ? lane : total - 1, qn);
      CandRec<R> nx = {};
      if (lane < total) nx = get_cand<R>(E.crec, kbase + (size_t)jn * kTile + qn);
      uint32_t n_proc[3] = {0u, 0u, 0u};
      for (uint32_t c0 = 0; c0 < total; c0 += 32) {
        const uint32_t ce = c0 + lane;
        const int j = jn;
        const uint32_t q = qn;
        const CandRec<R> cr = nx;
        if (c0 + 32 < total) {
          const uint32_t cn = ce + 32;
          jn = locate_event(cn < total ? cn : total - 1, qn);
          if (cn < total) nx = get_cand<R>(E.crec, kbase + (size_t)jn * kTile + qn);
        }
        int proc = 3, kx = 0;
        R u[4] = {0, 0, 0, 0}, eps = 0;
        if (ce < total) {
          const R s1 = cr.vx * cr.vx + cr.vy * cr.vy + cr.vz * cr.vz;
          const R v1 = r_sqrt(s1);
          const uint4 rr = philox4x32_10(make_uint4(cr.id, step, ctr2, 0u), key0, key1);
          proc = choose_process<R>(P, vlim, v1, s1, rr, s_acc, u, eps, kx);
          if (proc == 3 && dep)  // null: the velocity is kept
            deposit(rho_e, cr.cell, cr.off, fixed_charge(beta_of(v1, vlim) * cr.wj, wscale));
        }
        const uint32_t be = __ballot_sync(0xFFFFFFFFu, proc == 0);
        const uint32_t bn = __ballot_sync(0xFFFFFFFFu, proc == 1 || proc == 2);
        const uint32_t bi = __ballot_sync(0xFFFFFFFFu, proc == 2);
        n_proc[0] += __popc(be);
        n_proc[1] += __popc(bn & ~bi);
        n_proc[2] += __popc(bi);
        warp_births += __popc(bi);
        const uint32_t idx = pack_idx((uint32_t)j, q, cr.slot);
        if (proc == 0) {
          const uint32_t i = (e_tail + __popc(be & lanemask_lt)) & (kQ - 1);
          Q.e_idx[i] = idx;
          Q.e_cell[i] = cr.cell;
          Q.e_off[i] = cr.off;
          Q.e_wj[i] = cr.wj;
          Q.e_vx[i] = cr.vx;
          Q.e_vy[i] = cr.vy;
          Q.e_vz[i] = cr.vz;
          Q.e_eps[i] = eps;
          Q.e_u2[i] = u[2];
          Q.e_u3[i] = u[3];
        } else if (proc != 3) {
          const uint32_t i = (n_tail + __popc(bn & lanemask_lt)) & (kQ - 1);
          Q.n_idx[i] = idx;
          Q.n_id[i] = cr.id;
          Q.n_k[i] = (uint32_t)kx;
          Q.n_cell[i] = cr.cell;
          Q.n_off[i] = cr.off;
          Q.n_wj[i] = cr.wj;
          Q.n_eps[i] = eps;
          Q.n_u2[i] = u[2];
          Q.n_u3[i] = u[3];
        }
        e_tail += __popc(be);
        n_tail += __popc(bn);
        __syncwarp();
        if (e_tail - e_head >= 32u) drain_elastic(32u);
        if (n_tail - n_head >= 32u) drain_inelastic(32u);
      }
      if (e_tail != e_head) drain_elastic(e_tail - e_head);
      if (n_tail != n_head) drain_inelastic(n_tail - n_head);
      __syncwarp();
      // the warp's candidates and collisions, counted once
      if (lane == 0) {
        atomicAdd(&s_acc[ACC_CAND], (unsigned long long)total);
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (n_proc[k]) atomicAdd(&s_acc[ACC_COLL0 + k], (unsigned long long)n_proc[k]);
      }
    } else if (ion_chunk) {
      warp_births = total;
    }
    if (lane == 0) s_births[warp] = warp_births;
    __syncthreads();

    // ---- the chunk's slots: ordered scan over the instance's chunks ----------
    if (warp == 0) {
      uint32_t agg = 0;
      for (int w = 0; w < kCollWarps; ++w) agg += s_births[w];
      const uint32_t pre = chunk_lookback(r.coll_scan, c, first, agg, epoch, ctrl);
      if (lane == 0) s_prefix = pre;
    }
    __syncthreads();
    uint32_t off_w = s_prefix;
    for (int w = 0; w < warp; ++w) off_w += s_births[w];

    // ---- pass 2: write the births to their slots -----------------------------
    if (warp_births) {
      const uint32_t app_e = tail_slot(E, se), app_i = tail_slot(I, si);
      const uint32_t cap_e = E.cap_tiles * (uint32_t)kTile, cap_i = I.cap_tiles * (uint32_t)kTile;
      const SoAT<R> mi = soa_as<R>(I.buf[si.cur]);
      if (!ion_chunk) {
        // the ionized candidates in candidate order, queued (in the elastic
        // queue's index array, free after pass 1) and placed 32 at a time:
        // the n-th of the warp gets rank off_w + n
        uint32_t* bq = reinterpret_cast<CollQueues<R>*>(coll_smem)[warp].e_idx;
        const CandRec<R>* crec = reinterpret_cast<const CandRec<R>*>(E.crec);
        const size_t kbase = (size_t)kw * kTile;
        uint32_t b_head = 0, b_tail = 0;
        auto drain_births = [&](uint32_t n) {
          const bool on = lane < n;
          const uint32_t ri = on ? bq[(b_head + lane) & (kQ - 1)] : 0u;
          __syncwarp();
          if (on) {
            const uint32_t rank = off_w + b_head + lane;
            const CandRec<R> cr = crec[kbase + ri];
            const uint32_t pe = app_e + rank, pi = app_i + rank;
            if (pe >= cap_e || pi >= cap_i) {
              atomicCAS(&ctrl->error, 0, kErrCapacity);
            } else {
              if (P.field_mode == 1)
                born_pair<R>(P, me, mi, pe, pi, cr.cell, cr.off, cr.wj, cr.id, step, cr.vx,
                             se.next_id + rank, si.next_id + rank);
              else
                born_pair<R, false>(P, me, mi, pe, pi, cr.cell, cr.off, cr.wj, cr.id, step, cr.vx,
                                    se.next_id + rank, si.next_id + rank);
            }
          }
          b_head += n;
        };
        // the slots (with the ionization mark) of the next round load meanwhile
        uint32_t qn;
        int jn = locate_event(lane < total ? lane : total - 1, qn);
        uint32_t an = lane < total ? crec[kbase + (size_t)jn * kTile + qn].slot : 0u;
        for (uint32_t c0 = 0; c0 < total && b_tail < warp_births; c0 += 32) {
          const uint32_t ce = c0 + lane;
          const int j = jn;
          const uint32_t q = qn, a = an;
          if (c0 + 32 < total) {
            const uint32_t cn = ce + 32;
            jn = locate_event(cn < total ? cn : total - 1, qn);
            an = cn < total ? crec[kbase + (size_t)jn * kTile + qn].slot : 0u;
          }
          const bool ionized = ce < total && (a & kIonizedMark);
          const uint32_t b = __ballot_sync(0xFFFFFFFFu, ionized);
          if (ionized) bq[(b_tail + __popc(b & lanemask_lt)) & (kQ - 1)] = (uint32_t)j * kTile + q;
          b_tail += __popc(b);
          __syncwarp();
          if (b_tail - b_head >= 32u) drain_births(32u);
        }
        if (b_tail != b_head) drain_births(b_tail - b_head);
      } else {
        // electrons emitted at the cathode, after every ionization electron
        const SoAT<R> sb = soa_as<R>(E.stage_b);
        for (uint32_t c0 = 0; c0 < total; c0 += 32) {
          const uint32_t ce = c0 + lane;
          uint32_t q;
          const int j = locate_event(ce < total ? ce : total - 1, q);
          if (ce >= total) continue;
          const uint32_t rank = off_w + ce;
          const uint32_t pe = app_e + rank;
          if (pe >= cap_e) {
            atomicCAS(&ctrl->error, 0, kErrCapacity);
            continue;
          }
          const size_t o = (size_t)(kw + j) * kTile + q;
          write_marker(me, pe, sb.cell[o], sb.off[o], sb.vx[o], sb.vy[o], sb.vz[o], sb.wj[o],
                       kGenBit | ((se.next_id + rank) & kSerialMask));
        }
      }
    }
    __syncthreads();
  }
  if (cur_inst >= 0 && threadIdx.x < ACC_COUNT && s_acc[threadIdx.x])
    atomicAdd(r.inst[cur_inst].acc + threadIdx.x, s_acc[threadIdx.x]);
}

void launch_collide(const DeviceRefs& r, int grid, cudaStream_t s) {
  if (r.fp64)
    launch_step_kernel(k_collide<double>, grid, kCollThreads,
                       kCollWarps * sizeof(CollQueues<double>), s, r);
  else
    launch_step_kernel(k_collide<float>, grid, kCollThreads,
                       kCollWarps * sizeof(CollQueues<float>), s, r);
}

// The collision queues' shared memory (above the static 48 KB in FP64).
int collide_config() {
  cudaError_t e = cudaFuncSetAttribute(k_collide<float>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(kCollWarps * sizeof(CollQueues<float>)));
  if (e != cudaSuccess) return (int)e;
  e = cudaFuncSetAttribute(k_collide<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kCollWarps * sizeof(CollQueues<double>)));
  return (int)e;
}

static_assert(kCollThreads == 32 * kCollWarps, "kCollWarps warps per chunk");
static_assert(kCollMaxChunkTiles / kCollWarps <= 32, "per-tile counts live one per lane");
static_assert(kTile <= 128 && kCollMaxChunkTiles / kCollWarps <= 32,
              "pack_idx: 5 bits of tile, 7 of rank, 7 of slot");
static_assert((kCollMinChunkTiles & (kCollMinChunkTiles - 1)) == 0 &&
                  kCollMinChunkTiles % kCollWarps == 0,
              "chunk sizes are powers of two of whole warps");
static_assert((uint32_t)kTile < kIonizedMark, "candidate slots leave the top bit for the ionization mark");

}  // namespace slpic
