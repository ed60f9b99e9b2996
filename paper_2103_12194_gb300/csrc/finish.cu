// End of a step.  k_finish (one CTA per instance) updates the marker counts
// from the step's exact counters (the particle kernel compacted every tile,
// k_collide appended every birth), decides whether a store is repacked,
// publishes the step's deposit, solves the 1D Poisson equation for the next
// step's field (its exact integer sums) and commits the step's tallies; the
// last CTA plans the next step.  k_move evaluates the field from those sums
// over the whole grid and repacks the stores that became sparse.  With an imposed
// field the step deposits nothing and k_deposit forms the deposit from the
// markers when it is read.  Also: seeding, load validation and the Philox
// self-check kernel.
#include <algorithm>

#include "device_common.cuh"
#include "slpic_internal.h"
#include "step_ops.cuh"

namespace slpic {

namespace {

constexpr int kMoveThreads = 256;

// Segments a single warp plans (kPlanPerLane consecutive ones per lane; an
// instance's two segments stay in one lane).
constexpr int kPlanPerLane = 8;

__device__ __forceinline__ long long warp_incl_scan(long long v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// Write the plan's totals and reset the step's counters (one thread).
__device__ __forceinline__ void plan_totals(const DeviceRefs& r, int n_seg, unsigned int start,
                                            unsigned int wstart, unsigned int move,
                                            unsigned int coll) {
  r.seg_start[n_seg] = start;
  r.seg_wstart[n_seg] = wstart;
  r.coll_start[r.n_inst] = coll;
  r.move_start[n_seg] = move;
  r.ctrl->n_super = start;
  r.ctrl->w_total = wstart;
  r.ctrl->n_seg = n_seg;
  r.ctrl->n_coll_chunks = coll;
  r.ctrl->coll_counter = 0;
  r.ctrl->n_move_chunks = move;
  r.ctrl->move_counter = 0;
  r.ctrl->epoch = (r.ctrl->epoch + 1u) & 0x3FFFFFFFu;
  r.ctrl->finish_done = 0;
}

// The plan below by one warp (n_seg <= 32 kPlanPerLane), with shuffle scans
// and no block barrier.
__device__ void plan_next_warp(const DeviceRefs& r) {
  const int lane = threadIdx.x & 31;
  const int n_seg = r.n_inst * 2;
  const long long W = r.push_warps;
  long long ns[kPlanPerLane], w[kPlanPerLane], mv[kPlanPerLane], nc[kPlanPerLane / 2];
  long long s_ns = 0, s_w = 0, s_mv = 0, s_nc = 0;
#pragma unroll
  for (int j = 0; j < kPlanPerLane; ++j) {
    const int sg = lane * kPlanPerLane + j;
    ns[j] = w[j] = mv[j] = 0;
    if (sg < n_seg) {
      ns[j] = ((long long)r.sstate[sg].n_tiles + W - 1) / W;
      w[j] = ns[j] * ((sg & 1) ? kWeightIon : kWeightElectron);
      const Transfer& x = r.xfer[sg];
      if (x.compact) mv[j] = ((long long)x.n_tiles_old + kMoveChunkTiles - 1) / kMoveChunkTiles;
    }
    s_ns += ns[j];
    s_w += w[j];
    s_mv += mv[j];
  }
#pragma unroll
  for (int j = 0; j < kPlanPerLane / 2; ++j) {
    const int i = lane * (kPlanPerLane / 2) + j;
    nc[j] = 0;
    if (i < r.n_inst) {
      const long long T = r.coll_tiles[i];
      nc[j] = ((long long)r.sstate[2 * i].n_tiles + T - 1) / T +
              ((long long)r.sstate[2 * i + 1].n_tiles + kCollMaxChunkTiles - 1) /
                  kCollMaxChunkTiles;
    }
    s_nc += nc[j];
  }
  const long long i_ns = warp_incl_scan(s_ns, lane), i_w = warp_incl_scan(s_w, lane);
  const long long i_mv = warp_incl_scan(s_mv, lane), i_nc = warp_incl_scan(s_nc, lane);
  long long e_ns = i_ns - s_ns, e_w = i_w - s_w, e_mv = i_mv - s_mv, e_nc = i_nc - s_nc;
#pragma unroll
  for (int j = 0; j < kPlanPerLane; ++j) {
    const int sg = lane * kPlanPerLane + j;
    if (sg < n_seg) {
      r.seg_start[sg] = (unsigned int)e_ns;
      r.seg_wstart[sg] = (unsigned int)e_w;
      r.move_start[sg] = (unsigned int)e_mv;
    }
    e_ns += ns[j];
    e_w += w[j];
    e_mv += mv[j];
  }
#pragma unroll
  for (int j = 0; j < kPlanPerLane / 2; ++j) {
    const int i = lane * (kPlanPerLane / 2) + j;
    if (i < r.n_inst) r.coll_start[i] = (unsigned int)e_nc;
    e_nc += nc[j];
  }
  if (lane == 31)
    plan_totals(r, n_seg, (unsigned int)i_ns, (unsigned int)i_w, (unsigned int)i_mv,
                (unsigned int)i_nc);
}

// Plan the next step from the tiles in use (all threads of one CTA):
// particle-kernel super-tiles (push_warps tiles each) and their weights per
// segment, repacking chunks per segment and collision chunks per instance,
// as exclusive block scans in rounds of kFinThreads entries.
__device__ void plan_next(const DeviceRefs& r, long long* s_buf) {
  __shared__ long long s_carry[4];
  const int n_seg = r.n_inst * 2;
  if (n_seg <= 32 * kPlanPerLane) {
    if (threadIdx.x < 32) plan_next_warp(r);
    return;
  }
  const long long W = r.push_warps;
  const int t = threadIdx.x;
  if (t < 4) s_carry[t] = 0;
  __syncthreads();
  for (int base = 0; base < n_seg; base += kFinThreads) {
    const int sg = base + t;
    long long ns = 0, w = 0, mv = 0;
    if (sg < n_seg) {
      ns = ((long long)r.sstate[sg].n_tiles + W - 1) / W;
      w = ns * ((sg & 1) ? kWeightIon : kWeightElectron);
      const Transfer& x = r.xfer[sg];
      if (x.compact) mv = ((long long)x.n_tiles_old + kMoveChunkTiles - 1) / kMoveChunkTiles;
    }
    const long long i_ns = block_incl_scan<long long>(ns, s_buf);
    const long long i_w = block_incl_scan<long long>(w, s_buf);
    const long long i_mv = block_incl_scan<long long>(mv, s_buf);
    if (sg < n_seg) {
      r.seg_start[sg] = (unsigned int)(s_carry[0] + i_ns - ns);
      r.seg_wstart[sg] = (unsigned int)(s_carry[1] + i_w - w);
      r.move_start[sg] = (unsigned int)(s_carry[2] + i_mv - mv);
    }
    __syncthreads();
    if (t == kFinThreads - 1) {
      s_carry[0] += i_ns;
      s_carry[1] += i_w;
      s_carry[2] += i_mv;
    }
    __syncthreads();
  }
  for (int base = 0; base < r.n_inst; base += kFinThreads) {
    const int i = base + t;
    long long nc = 0;
    if (i < r.n_inst) {
      const long long T = r.coll_tiles[i];
      nc = ((long long)r.sstate[2 * i].n_tiles + T - 1) / T +
           ((long long)r.sstate[2 * i + 1].n_tiles + kCollMaxChunkTiles - 1) / kCollMaxChunkTiles;
    }
    const long long i_nc = block_incl_scan<long long>(nc, s_buf);
    if (i < r.n_inst) r.coll_start[i] = (unsigned int)(s_carry[3] + i_nc - nc);
    __syncthreads();
    if (t == kFinThreads - 1) s_carry[3] += i_nc;
    __syncthreads();
  }
  if (t == 0)
    plan_totals(r, n_seg, (unsigned int)s_carry[0], (unsigned int)s_carry[1],
                (unsigned int)s_carry[2], (unsigned int)s_carry[3]);
}

}  // namespace

// mode 0: finish a step (one CTA per instance; the last one plans the next
// step); mode 1: plan only (one CTA).  Dynamic shared memory: net_nodes
// int64 nodes for the net deposit (0: read it from global memory).
__global__ void __launch_bounds__(kFinThreads) k_finish(DeviceRefs r, int mode, int net_nodes) {
  extern __shared__ long long s_dyn[];
  __shared__ long long s_i64[32];
  __shared__ __int128 s_i128[32];
  __shared__ unsigned long long s_acc[ACC_COUNT];
  __shared__ int s_flag;
  step_kernel_entry();
  Control* ctrl = r.ctrl;
  const int t = threadIdx.x;
  if (mode == 1) {
    for (int sg = t; sg < 2 * r.n_inst; sg += kFinThreads) r.xfer[sg].compact = 0;
    __syncthreads();
    plan_next(r, s_i64);
    return;
  }
  if (*((volatile int*)&ctrl->error)) return;
  const int inst = blockIdx.x;
  const InstDev& P = r.inst[inst];
  InstState& is = r.istate[inst];
  unsigned long long* a = P.acc;
  const int N = P.n_cells, nn = N + 1;
  long long* s_net = nn <= net_nodes ? s_dyn : nullptr;

  // ---- accumulators and the step's deposit, all threads at once -------------
  // deposit -> rho_last (and the net charge to shared memory); clear both
  if (t < ACC_COUNT) {
    s_acc[t] = a[t];
    a[t] = 0ull;
  }
  // (with an imposed field nothing was deposited: the deposit is formed from
  // the markers when it is read)
  // (four nodes per thread at a time: their loads are issued before any store)
  for (int k0 = t; k0 < nn && P.field_mode == 1; k0 += 4 * kFinThreads) {
    long long qe[4], qi[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k0 + u * kFinThreads;
      qe[u] = k < nn ? (long long)P.rho_acc[kElectron][k] : 0ll;
      qi[u] = k < nn ? (long long)P.rho_acc[kIon][k] : 0ll;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k0 + u * kFinThreads;
      if (k >= nn) break;
      P.rho_last[kElectron][k] = qe[u];
      P.rho_last[kIon][k] = qi[u];
      P.rho_acc[kElectron][k] = 0ull;
      P.rho_acc[kIon][k] = 0ull;
      if (s_net) s_net[k] = qi[u] - qe[u];
    }
  }
  __syncthreads();

  // ---- marker counts and where the stores end (one thread per species) -------
  // survivors = live - absorbed; births (ionizations: an electron and an ion
  // each; emitted electrons) were appended after the last live marker
  if (t < 2) {
    const int sp = t;
    const uint32_t n_ionz = (uint32_t)s_acc[ACC_COLL2], n_see = (uint32_t)s_acc[ACC_SEE];
    SpeciesState& st = r.sstate[inst * 2 + sp];
    const SpeciesDev& S = P.sp[sp];
    Transfer& x = r.xfer[inst * 2 + sp];
    const uint32_t absorbed = (uint32_t)(s_acc[ACC_NABS + 2 * sp] + s_acc[ACC_NABS + 2 * sp + 1]);
    const uint32_t nb = sp ? n_ionz : n_ionz + n_see;
    const SpeciesState s0 = st;
    const uint32_t surv = s0.n_live - absorbed;
    const uint32_t tail =
        s0.n_tiles ? (s0.n_tiles - 1) * (uint32_t)kTile + S.fill[s0.cur][s0.n_tiles - 1] : 0u;
    const uint32_t end = tail + nb;
    const uint32_t n_new = surv + nb;
    const uint32_t nt = (end + kTile - 1) / kTile;
    // repack when under 15/16 of the slots in use are live: tiles with holes
    // cost the particle kernel nearly as much as full ones, and a growing
    // avalanche leaves many (at 3/4 a 1000-step run of the benchmark ran at
    // half the rate in its last steps)
    const uint32_t compact =
        (nt > 2 && (unsigned long long)n_new * 16 < (unsigned long long)nt * kTile * 15) ? 1u : 0u;
    x.compact = compact;
    x.src = s0.cur;
    x.dst = compact ? s0.cur ^ 1u : s0.cur;
    x.n_tiles_old = nt;
    x.n_new = n_new;
    x.tail = tail;
    x.end = end;
    if (sp == kElectron) {
      // electron collision chunks of the next step: the largest power of two
      // (tiles) with about kCollTargetPerWarp candidates per warp at this
      // step's candidates per tile
      const unsigned long long cand = s_acc[ACC_CAND];
      const unsigned long long room =
          cand ? (unsigned long long)kCollTargetPerWarp * kCollWarps * s0.n_tiles / cand
               : (unsigned long long)kCollMaxChunkTiles;
      unsigned int T = kCollMaxChunkTiles;
      while (T > (unsigned int)kCollMinChunkTiles && T > room) T >>= 1;
      r.coll_tiles[inst] = T;
    }
    SpeciesState s1;
    s1.cur = x.dst;
    s1.n_live = n_new;
    s1.next_id = s0.next_id + nb;
    s1.n_tiles = compact ? (n_new + kTile - 1) / kTile : nt;
    st = s1;
  }
  __syncthreads();
  // fills of the tail tile and the new tiles: their slots below `end` are live
  // (k_move reads them when it repacks the store)
  for (int sp = 0; sp < 2; ++sp) {
    const SpeciesDev& S = P.sp[sp];
    const Transfer& x = r.xfer[inst * 2 + sp];
    if (x.end == x.tail) continue;
    for (uint32_t k = x.tail / kTile + t; k < x.n_tiles_old; k += kFinThreads)
      S.fill[x.src][k] = min(x.end - k * (uint32_t)kTile, (uint32_t)kTile);
  }

  // ---- Poisson: (phi[k+1] - 2 phi[k] + phi[k-1]) = -C net_k, k = 1..N-1 ----
  // With D_k = phi[k] - phi[k-1]: D_k = D_1 - C I_k, I_k = sum_{0<j<k} net_j,
  // and phi[N] = V fixes D_1 = (V + C J_N) / N, J_N = sum_{0<i<=N} I_i.
  // The node field is the centred difference of phi, written with the exact
  // integer sums: E_k = -(D_k + D_{k+1}) / (2 dx) = -(2 D_1 - C (I_k + I_{k+1}))
  // / (2 dx), one-sided at the electrodes.  This CTA leaves I_k and D_1; k_move,
  // which follows every step on many SMs, evaluates E in FP64 (poisson_field),
  // and phi is formed on demand (k_phi) when it is read.
  if (P.field_mode == 1) {
    const int chunk = (N + kFinThreads - 1) / kFinThreads;  // over k = 1..N
    const int k0 = 1 + t * chunk;
    long long I0;
    const double D1 = poisson_d1(P, s_net, k0, chunk, s_i64, s_i128, &I0);
    long long Ik = I0;
    for (int k = k0; k < k0 + chunk && k <= N; ++k) {
      P.pois_I[k] = Ik;
      if (k <= N - 1) Ik += net_at(P, s_net, k);
    }
    if (t == 0) *P.pois_D1 = D1;
  }

  // ---- tallies: one thread per 8-byte slot of the record ---------------------
  if (t < kTallySlots)
    commit_tally_slot(P, t, s_acc, is.step, is.n_steps_done, r.sstate[inst * 2].n_live,
                      r.sstate[inst * 2 + 1].n_live, is.w_live, &is.ion_steps);
  __syncthreads();
  if (t == 0) {
    is.step += 1u;
    is.n_steps_done += 1;
  }

  // ---- the last CTA plans the next step --------------------------------------
  __threadfence();
  __syncthreads();
  if (t == 0) {
    const unsigned int ticket = atomicAdd(&ctrl->finish_done, 1u);
    s_flag = ticket == gridDim.x - 1 ? 1 : 0;
  }
  __syncthreads();
  if (s_flag) {
    __threadfence();
    plan_next(r, s_i64);
  }
}

// The deposit of instance inst's live markers into its last-step grids
// (zeroed by the caller): each marker adds fixed_charge(beta(|v|) w_j) at its
// position, as the step deposits it.  A step's deposit is a function of the
// markers after it, so with an imposed field it is formed here, when read,
// instead of during every step.  One warp per tile, tiles of both species in
// a grid-stride loop.
template <typename R>
__global__ void __launch_bounds__(256) k_deposit(DeviceRefs r, int inst) {
  const InstDev& P = r.inst[inst];
  const StepConsts<R>& K = consts<R>(P);
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int n_warps = (gridDim.x * blockDim.x) >> 5;
  const SpeciesState se = r.sstate[inst * 2], si = r.sstate[inst * 2 + 1];
  const uint32_t ne = se.n_tiles, n_items = se.n_tiles + si.n_tiles;
  for (uint32_t it = warp; it < n_items; it += n_warps) {
    const int sp = it < ne ? 0 : 1;
    const uint32_t k = it < ne ? it : it - ne;
    const SpeciesState& st = sp ? si : se;
    const SoAT<R> m = soa_as<R>(P.sp[sp].buf[st.cur]);
    const R vlim = K.vlim[sp];
    const bool limited = vlim < (R)INFINITY;
    unsigned long long* rho = reinterpret_cast<unsigned long long*>(P.rho_last[sp]);
    const uint32_t n = P.sp[sp].fill[st.cur][k];
    for (uint32_t i = lane; i < n; i += 32) {
      const size_t o = (size_t)k * kTile + i;
      const R vx = m.vx[o], vy = m.vy[o], vz = m.vz[o];
      const R b = limited ? beta_of(r_sqrt(vx * vx + vy * vy + vz * vz), vlim) : (R)1;
      deposit(rho, m.cell[o], m.off[o], fixed_charge(b * m.wj[o], K.wscale));
    }
  }
}

void launch_deposit(const DeviceRefs& r, int inst, int n_tiles, cudaStream_t s) {
  const int grid = std::max(1, std::min((n_tiles + 7) / 8, 4096));
  if (r.fp64) k_deposit<double><<<grid, 256, 0, s>>>(r, inst);
  else k_deposit<float><<<grid, 256, 0, s>>>(r, inst);
}

// phi_k = k D_1 - C J_k, J_k = sum_{0<i<=k} I_i, from the last step's deposit
// (one CTA; read only when the field is read).
__global__ void __launch_bounds__(kFinThreads) k_phi(DeviceRefs r, int inst) {
  __shared__ long long s_i64[32];
  __shared__ __int128 s_i128[32];
  const InstDev& P = r.inst[inst];
  const int N = P.n_cells;
  const int chunk = (N + kFinThreads - 1) / kFinThreads;
  const int k0 = 1 + threadIdx.x * chunk;
  long long Ik;
  const double D1 = poisson_d1(P, nullptr, k0, chunk, s_i64, s_i128, &Ik);
  const double C = P.pois_C;
  // J at the chunk start: exclusive scan of the chunks' sums of I
  __int128 locJ = 0;
  {
    long long I = Ik;
    for (int k = k0; k < k0 + chunk && k <= N; ++k) {
      locJ += (__int128)I;
      if (k <= N - 1) I += P.rho_last[kIon][k] - P.rho_last[kElectron][k];
    }
  }
  const __int128 incJ = block_incl_scan<__int128>(locJ, s_i128);
  __int128 J = incJ - locJ;
  for (int k = k0; k < k0 + chunk && k <= N; ++k) {
    J += (__int128)Ik;
    if (k <= N - 1) Ik += P.rho_last[kIon][k] - P.rho_last[kElectron][k];
    P.phi[k] = k == N ? P.V : (double)k * D1 - C * (double)J;
  }
  if (threadIdx.x == 0) P.phi[0] = 0.0;
}

void launch_phi(const DeviceRefs& r, int inst, cudaStream_t s) {
  k_phi<<<1, kFinThreads, 0, s>>>(r, inst);
}

// Dynamic shared memory of k_finish: the net deposit of the largest grid,
// when it fits (DeviceRefs::finish_net_nodes, from finish_config).
int finish_config(int max_nodes, int* net_nodes) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return (int)e;
  const int room = (optin - 8 * 1024) / 8;  // static shared memory stays below 8 KB
  *net_nodes = max_nodes <= room ? max_nodes : 0;
  // the limit is the most a CTA can have, so that one context's
  // configuration never lowers it under another's
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, k_finish);
  if (e != cudaSuccess) return (int)e;
  e = cudaFuncSetAttribute(k_finish, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes);
  return (int)e;
}

void launch_finish(const DeviceRefs& r, int mode, cudaStream_t s) {
  const int grid = mode == 1 ? 1 : r.n_inst;
  const int nodes = mode == 1 ? 0 : r.finish_net_nodes;
  launch_step_kernel(k_finish, grid, kFinThreads, (size_t)nodes * 8, s, r, mode, nodes);
}

// ---------------------------------------------------------------------------
// Repacking of the stores k_finish marked sparse: chunks of kMoveChunkTiles
// tiles, handed out in order; each chunk's destination is the prefix of the
// fills of the tiles before it (ordered scan with decoupled look-back); the
// live markers keep their order.  The chunk also writes the fills of the
// repacked store for the tiles with its indices.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kMoveThreads) k_move(DeviceRefs r) {
  __shared__ uint32_t s_fill[kMoveChunkTiles];
  __shared__ uint32_t s_pre[kMoveChunkTiles];
  __shared__ unsigned int s_chunk;
  constexpr int kPerLaneTiles = kMoveChunkTiles / 32;
  step_kernel_entry();
  Control* ctrl = r.ctrl;
  if (*((volatile int*)&ctrl->error)) return;
  // the field of the step's Poisson solves: CTA b takes part b / n_inst of
  // instance b % n_inst (every instance gets gridDim / n_inst CTAs, at least
  // one), node by node
  {
    const int n_inst = r.n_inst;
    const int parts = max(1, (int)gridDim.x / n_inst);
    for (int b = blockIdx.x; b < n_inst * parts; b += gridDim.x) {
      const InstDev& P = r.inst[b % n_inst];
      if (P.field_mode == 1)
        poisson_field(P, (b / n_inst) * blockDim.x + threadIdx.x, parts * blockDim.x);
    }
  }
  const unsigned int n_chunks = ctrl->n_move_chunks;
  if (n_chunks == 0) return;
  const unsigned int epoch = ctrl->epoch;
  const int n_seg = r.n_inst * 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_chunk = atomicAdd(&ctrl->move_counter, 1u);
    __syncthreads();
    const unsigned int c = s_chunk;
    if (c >= n_chunks) break;
    int seg = 0;
    {
      int lo = 0, hi = n_seg - 1;  // last segment with move_start <= c
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (r.move_start[mid] <= c) lo = mid;
        else hi = mid - 1;
      }
      seg = lo;
    }
    const Transfer& x = r.xfer[seg];
    const SpeciesDev& S = r.inst[seg >> 1].sp[seg & 1];
    const unsigned int first = r.move_start[seg];
    const uint32_t k0 = (c - first) * kMoveChunkTiles;
    for (int j = threadIdx.x; j < kMoveChunkTiles; j += kMoveThreads) {
      const uint32_t k = k0 + j;
      s_fill[j] = k < x.n_tiles_old ? S.fill[x.src][k] : 0u;
    }
    __syncthreads();
    if (warp == 0) {
      // lane l sums tiles l * kPerLaneTiles ..; scan over the lanes
      uint32_t loc = 0;
      for (int j = 0; j < kPerLaneTiles; ++j) loc += s_fill[lane * kPerLaneTiles + j];
      uint32_t inc = loc;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t n = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += n;
      }
      const uint32_t agg = __shfl_sync(0xFFFFFFFFu, inc, 31);
      const uint32_t excl = chunk_lookback(r.move_scan, c, first, agg, epoch, ctrl);
      uint32_t run = excl + inc - loc;
      for (int j = 0; j < kPerLaneTiles; ++j) {
        s_pre[lane * kPerLaneTiles + j] = run;
        run += s_fill[lane * kPerLaneTiles + j];
      }
    }
    __syncthreads();
    // one warp per tile, in order of the tiles
    const SoAT<R> src = soa_as<R>(S.buf[x.src]), dst = soa_as<R>(S.buf[x.dst]);
    for (int j = warp; j < kMoveChunkTiles; j += kMoveThreads / 32) {
      const uint32_t n = s_fill[j];
      const size_t from = (size_t)(k0 + j) * kTile, to = s_pre[j];
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
    // fills of the repacked store: full tiles, the last one partial
    const uint32_t nt_new = (x.n_new + kTile - 1) / kTile;
    for (int j = threadIdx.x; j < kMoveChunkTiles; j += kMoveThreads) {
      const uint32_t k = k0 + j;
      if (k < nt_new) S.fill[x.dst][k] = min(x.n_new - k * (uint32_t)kTile, (uint32_t)kTile);
    }
    __syncthreads();
  }
}

void launch_move(const DeviceRefs& r, int grid, cudaStream_t s) {
  if (r.fp64) launch_step_kernel(k_move<double>, grid, kMoveThreads, 0, s, r);
  else launch_step_kernel(k_move<float>, grid, kMoveThreads, 0, s, r);
}

// ---------------------------------------------------------------------------
// Seeding: n markers appended at index base = n_live of the species, drawn
// from Philox with counter (id, 0xFFFFFFFF, inst * 2 + species, block).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_seed(DeviceRefs r, int inst, int sp, uint32_t base, uint32_t first_id,
                       uint32_t n, int mode, double ekin_d, double elo_d, double lr_d,
                       double wj_d) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const InstDev& P = r.inst[inst];
  const SpeciesDev& S = P.sp[sp];
  const StepConsts<R>& K = consts<R>(P);
  const SoAT<R> d = soa_as<R>(S.buf[r.sstate[inst * 2 + sp].cur]);
  const R ekin = (R)ekin_d, elo = (R)elo_d, lr = (R)lr_d, wj = (R)wj_d;
  const uint32_t id = first_id + i;
  R u[4];
  uniform4<R>(philox4x32_10(make_uint4(id, kSeedStep, P.ctr_inst * 2u + (uint32_t)sp, 0u),
                            P.key0, P.key1),
              u);
  int cell = 0;
  R off = (R)0, vx = (R)0, vy = (R)0, vz = (R)0;
  const int N = P.n_cells;
  if (mode == 0) {
    off = u[0];
    const R v = r_sqrt(ekin * K.K_V[sp]);
    const R ct = u[1];
    const R st = r_sqrt(r_max((R)0, ((R)1 - ct) * ((R)1 + ct)));
    const R ph = K.two_pi * u[2];
    vx = v * ct;
    vy = v * (st * r_cos(ph));
    vz = v * (st * r_sin(ph));
  } else if (mode == 2 || mode == 3) {
    const R p = u[0] * (R)N;
    const R fl = r_floor(p);
    cell = (int)fl;
    off = p - fl;
    if (cell >= N) {
      cell = N - 1;
      off = nextafter_below_one<R>();
    }
    if (mode == 2) {
      const R e = elo * r_exp(u[1] * lr);
      isotropic(r_sqrt(e * K.K_V[sp]), u[2], u[3], K.two_pi, vx, vy, vz);
    } else {
      R g[4];
      uniform4<R>(philox4x32_10(make_uint4(id, kSeedStep, P.ctr_inst * 2u + (uint32_t)sp, 1u),
                                P.key0, P.key1),
                  g);
      // gas-temperature Maxwellian of this species
      const R sig = ekin;  // sqrt(k T / m), passed in ekin for this mode
      const R r1 = r_sqrt((R)-2 * r_log(u[1]));
      const R r2 = r_sqrt((R)-2 * r_log(u[3]));
      const R a1 = K.two_pi * u[2], a2 = K.two_pi * g[0];
      vx = sig * (r1 * r_cos(a1));
      vy = sig * (r1 * r_sin(a1));
      vz = sig * (r2 * r_cos(a2));
    }
  }
  const uint32_t o = base + i;
  d.cell[o] = cell;
  d.off[o] = off;
  d.vx[o] = vx;
  d.vy[o] = vy;
  d.vz[o] = vz;
  d.wj[o] = wj;
  d.id[o] = id & kSerialMask;
}

void launch_seed(const DeviceRefs& r, int inst, int species, uint32_t base, uint32_t first_id,
                 uint32_t n, int mode, double e0, double e_lo, double lr, double wj,
                 cudaStream_t s) {
  if (n == 0) return;
  const int threads = 256;
  const unsigned int grid = (n + threads - 1) / threads;
  if (r.fp64)
    k_seed<double><<<grid, threads, 0, s>>>(r, inst, species, base, first_id, n, mode, e0, e_lo,
                                           lr, wj);
  else
    k_seed<float><<<grid, threads, 0, s>>>(r, inst, species, base, first_id, n, mode, e0, e_lo,
                                          lr, wj);
}

// Check loaded markers (cell in [0, N), offset in [0, 1), finite velocities,
// non-negative weight below 2^39 charge units); records the smallest bad index in *bad and the
// fixed-point sum of the weights in *wsum.
template <typename R>
__global__ void k_validate(SoA dv, uint32_t n, int N, int shift, unsigned int* bad,
                           unsigned long long* wsum) {
  const SoAT<R> d = soa_as<R>(dv);
  const R wscale = (R)ldexp(1.0, shift);  // 2^shift, exact
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long w = 0;
  if (i < n) {
    const R o = d.off[i], x = d.vx[i], y = d.vy[i], z = d.vz[i], wj = d.wj[i];
    const int c = d.cell[i];
    // the fixed-point weight must stay below 2^39 units so that the 24-bit
    // linear split of the deposit cannot overflow 64 bits
    const bool ok = c >= 0 && c < N && o >= (R)0 && o < (R)1 && isfinite(x) && isfinite(y) &&
                    isfinite(z) && wj >= (R)0 && wj * wscale < (R)549755813888.0;
    if (!ok) atomicMin(bad, i);
    else w = (unsigned long long)fixed_charge(wj, wscale);
  }
  for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xFFFFFFFFu, w, o);
  if ((threadIdx.x & 31) == 0 && w) atomicAdd(wsum, w);
}

void launch_validate(int fp64, const SoA& d, uint32_t n, int N, int shift, unsigned int* bad,
                     unsigned long long* wsum, cudaStream_t s) {
  if (n == 0) return;
  const int threads = 256;
  if (fp64)
    k_validate<double><<<(n + threads - 1) / threads, threads, 0, s>>>(d, n, N, shift, bad, wsum);
  else
    k_validate<float><<<(n + threads - 1) / threads, threads, 0, s>>>(d, n, N, shift, bad, wsum);
}

__global__ void k_philox(uint32_t k0, uint32_t k1, const uint4* ctr, uint4* out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox4x32_10(ctr[i], k0, k1);
}

__global__ void k_philox2(uint32_t k, const uint2* ctr, uint2* out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox2x32_10(ctr[i], k);
}

void launch_philox2(uint32_t k, const uint32_t* ctr, uint32_t* out, long long n,
                    cudaStream_t s) {
  if (n <= 0) return;
  const int threads = 256;
  const long long grid = (n + threads - 1) / threads;
  k_philox2<<<(unsigned int)grid, threads, 0, s>>>(k, reinterpret_cast<const uint2*>(ctr),
                                                   reinterpret_cast<uint2*>(out), n);
}

// Load the Philox kernel's module now (CUDA loads modules lazily, and the
// load can reserve device memory).
int philox_preload() {
  cudaFuncAttributes a;
  return (int)cudaFuncGetAttributes(&a, k_philox);
}

void launch_philox(uint32_t k0, uint32_t k1, const uint32_t* ctr, uint32_t* out, long long n,
                   cudaStream_t s) {
  if (n <= 0) return;
  const int threads = 256;
  const long long grid = (n + threads - 1) / threads;
  k_philox<<<(unsigned int)grid, threads, 0, s>>>(k0, k1, reinterpret_cast<const uint4*>(ctr),
                                                  reinterpret_cast<uint4*>(out), n);
}

}  // namespace slpic
