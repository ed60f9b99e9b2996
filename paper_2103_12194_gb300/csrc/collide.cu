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
// Work: chunks of kCollChunkTiles consecutive tiles (each warp kCollWarpTiles
// of them; the warp numbers the candidates of its tiles in (tile, slot) order
// and takes them 32 at a time, one lane each, reading each candidate's
// record -- its state and slot, one 32-byte sector in float -- and writing
// only the new velocity to its slot), handed out in order (electron
// tiles of an instance, then its ion tiles).  The births of a chunk (ionizations; for ion chunks the
// electrons the particle kernel staged for emission) get their slots from an
// ordered scan over the chunks (decoupled look-back), so they are appended
// after the last live marker in (tile, slot) order -- ionization electrons
// first, emitted electrons after -- with their final serial numbers, whatever
// the scheduling.
#include "device_common.cuh"
#include "slpic_internal.h"
#include "step_ops.cuh"

namespace slpic {

namespace {

constexpr int kCollThreads = 256;

}  // namespace

template <typename R>
__global__ void __launch_bounds__(kCollThreads, 4) k_collide(DeviceRefs r) {
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
    const unsigned int e_chunks = (se.n_tiles + kCollChunkTiles - 1) / kCollChunkTiles;
    const bool ion_chunk = local >= e_chunks;
    const uint32_t nt = ion_chunk ? si.n_tiles : se.n_tiles;
    // this warp's tiles: kCollWarpTiles consecutive ones, tile kw + j at lane j
    const uint32_t kw = (ion_chunk ? local - e_chunks : local) * kCollChunkTiles +
                        warp * kCollWarpTiles;
    const SoAT<R> me = soa_as<R>(E.buf[se.cur]);
    const StepConsts<R>& K = consts<R>(P);
    const R kv = K.K_V[kElectron], vlim = K.vlim[kElectron];
    // events of the tiles (electron chunks: queued candidates; ion chunks:
    // electrons emitted at the cathode) and their exclusive prefix: the
    // warp's events are numbered in (tile, slot) order
    uint32_t cnt = 0;
    if (lane < kCollWarpTiles && kw + lane < nt) cnt = ion_chunk ? I.births[kw + lane] : E.n_cand[kw + lane];
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
    // Rounds of 32 candidates, one per lane; the records of the next round are
    // read while this round scatters, so their load latency overlaps it.
    uint32_t warp_births = 0;
    if (!ion_chunk && total) {
      const uint32_t ctr2 = P.ctr_inst * 2u, key0 = P.key0, key1 = P.key1;
      const bool dep = P.field_mode == 1;  // imposed field: the deposit is formed when read
      unsigned long long* rho_e = P.rho_acc[kElectron];
      const R wscale = K.wscale;
      uint32_t qn;
      int jn = locate_event(lane < total ? lane : total - 1, qn);
      CandRec<R> nx = {};
      if (lane < total) nx = get_cand<R>(E.crec, (size_t)(kw + jn) * kTile + qn);
      uint32_t n_proc[3] = {0u, 0u, 0u};
      for (uint32_t c0 = 0; c0 < total; c0 += 32) {
        const uint32_t ce = c0 + lane;
        const int j = jn;
        const uint32_t q = qn;
        const CandRec<R> cr = nx;
        if (c0 + 32 < total) {
          const uint32_t cn = ce + 32;
          jn = locate_event(cn < total ? cn : total - 1, qn);
          if (cn < total) nx = get_cand<R>(E.crec, (size_t)(kw + jn) * kTile + qn);
        }
        bool ionized = false;
        int proc = 3;
        if (ce < total) {
          const size_t base = (size_t)(kw + j) * kTile;
          const size_t o = base + cr.slot;
          const uint32_t id = cr.id;
          R vx = cr.vx, vy = cr.vy, vz = cr.vz;
          const R s1 = vx * vx + vy * vy + vz * vz;
          const R v1 = r_sqrt(s1);
          const uint4 rr = philox4x32_10(make_uint4(id, step, ctr2, 0u), key0, key1);
          R es = (R)0;
          const Velocity<R> nv =
              collide<R>(P, kv, vlim, vx, vy, vz, v1, s1, rr, id, step, cr.wj, s_acc, &es, &proc);
          if (proc < 3) {
            vx = nv.vx;
            vy = nv.vy;
            vz = nv.vz;
            me.vx[o] = vx;
            me.vy[o] = vy;
            me.vz[o] = vz;
            if (proc == 2) {
              // mark for pass 2, with the secondary's energy in place of vx
              ionized = true;
              CandRec<R>* w = reinterpret_cast<CandRec<R>*>(E.crec) + base + q;
              w->slot = cr.slot | kIonizedMark;
              w->vx = es;
            }
          }
          if (dep)
            deposit(rho_e, cr.cell, cr.off,
                    fixed_charge(beta_of(r_sqrt(vx * vx + vy * vy + vz * vz), vlim) * cr.wj,
                                 wscale));
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) n_proc[k] += __popc(__ballot_sync(0xFFFFFFFFu, proc == k));
        warp_births += __popc(__ballot_sync(0xFFFFFFFFu, ionized));
      }
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
        uint32_t ranked = 0;
        for (uint32_t c0 = 0; c0 < total; c0 += 32) {
          const uint32_t ce = c0 + lane;
          uint32_t q;
          const int j = locate_event(ce < total ? ce : total - 1, q);
          const size_t base = (size_t)(kw + j) * kTile;
          const CandRec<R>* rp = reinterpret_cast<const CandRec<R>*>(E.crec) + base + q;
          const uint32_t a = ce < total ? rp->slot : 0u;
          const bool ionized = ce < total && (a & kIonizedMark);
          const uint32_t b = __ballot_sync(0xFFFFFFFFu, ionized);
          if (ionized) {
            const uint32_t rank = off_w + ranked + __popc(b & lanemask_lt);
            const CandRec<R> cr = *rp;
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
          ranked += __popc(b);
        }
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
  if (r.fp64) launch_step_kernel(k_collide<double>, grid, kCollThreads, 0, s, r);
  else launch_step_kernel(k_collide<float>, grid, kCollThreads, 0, s, r);
}

static_assert(kCollThreads == 32 * kCollWarps, "kCollWarps warps per chunk");
static_assert(kCollWarpTiles <= 32, "per-tile counts live one per lane");
static_assert((uint32_t)kTile < kIonizedMark, "candidate slots leave the top bit for the ionization mark");

}  // namespace slpic
