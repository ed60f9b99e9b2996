// Monte-Carlo collisions of the null-collision candidates queued by the
// particle kernel (Sec. III and IV), and the placement of every birth of the
// step.  For a candidate (an electron that drew u < P0 this step) the process
// is chosen by comparing u' P0 with the cumulative rates
// n_g sigma_k(eps) beta v dt (Eq. SLPICcollisionNumber with beta_n = 1,
// whole-marker collisions); elastic collisions scatter by the Vahedi-Surendra
// angles with the recoil loss, excitation removes its threshold and scatters
// isotropically, ionization shares the excess energy between the primary and
// a born electron and creates an Ar+ at the same position with the same flux
// weight.  Each candidate is then deposited with its new density weight.
//
// Work: chunks of kCollChunkTiles consecutive tiles (each warp kCollWarpTiles
// of them; the warp numbers the candidates of its tiles in (tile, slot) order
// and takes them 32 at a time, one lane each), handed out in order (electron
// tiles of an instance, then its ion tiles).  The births of a chunk (ionizations; for ion chunks the
// electrons the particle kernel staged for emission) get their slots from an
// ordered scan over the chunks (decoupled look-back), so they are appended
// after the last live marker in (tile, slot) order -- ionization electrons
// first, emitted electrons after -- with their final serial numbers, whatever
// the scheduling.
#include "device_common.cuh"
#include "slpic_internal.h"

namespace slpic {

namespace {

constexpr int kCollThreads = 256;

// Interpolated cumulative cross sections at eps (linear between the nodes of
// the octave-uniform grid, held constant outside it): xs[0 .. n_exc + 1].
// The node index and the fraction come exactly from the exponent and
// mantissa bits of eps.
__device__ __forceinline__ void xsec(const InstDev& P, float eps, float* xs) {
  const StepConsts<float>& K = P.c32;
  int j;
  float t;
  if (!(eps >= K.e_lo)) {
    j = 0;
    t = 0.0f;
  } else if (eps >= K.e_hi) {
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
  const int st = P.tab_stride;
  const float4 a = __ldg(P.table + j * st);
  const float4 c = __ldg(P.table + (j + 1) * st);
  xs[0] = a.x + t * (c.x - a.x);
  xs[1] = a.y + t * (c.y - a.y);
  xs[2] = a.z + t * (c.z - a.z);
  xs[3] = a.w + t * (c.w - a.w);
  if (st > 1) {
    const float4 a1 = __ldg(P.table + j * st + 1);
    const float4 c1 = __ldg(P.table + (j + 1) * st + 1);
    xs[4] = a1.x + t * (c1.x - a1.x);
  }
}

__device__ __forceinline__ void xsec(const InstDev& P, double eps, double* xs) {
  const StepConsts<double>& K = P.c64;
  int j;
  double t;
  if (!(eps >= K.e_lo)) {
    j = 0;
    t = 0.0;
  } else if (eps >= K.e_hi) {
    j = P.tab_nodes - 1;
    t = 0.0;
  } else {
    const unsigned long long b = (unsigned long long)__double_as_longlong(eps);
    const int octave = (int)(b >> 52) - 1023 - P.tab_lo_exp2;
    const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
    const int sh = 52 - P.tab_log2_sub;
    j = (octave << P.tab_log2_sub) + (int)(mant >> sh);
    const double scale = __longlong_as_double((long long)(1023 - sh) << 52);  // 2^-sh
    t = (double)(mant & ((1ull << sh) - 1ull)) * scale;
  }
  const TabNode64& a = P.table64[j];
  const TabNode64& c = P.table64[j + 1];
  const int n_proc = P.n_exc + 2;
#pragma unroll
  for (int k = 0; k < kMaxProc; ++k)
    if (k < n_proc) xs[k] = a.s[k] + t * (c.s[k] - a.s[k]);
}

template <typename R>
__device__ __forceinline__ void deposit(unsigned long long* rho, int cell, R off, long long Q) {
  const long long right = right_share(Q, off);
  const long long left = Q - right;
  if (left) atomicAdd(rho + cell, (unsigned long long)left);
  if (right) atomicAdd(rho + cell + 1, (unsigned long long)right);
}

template <typename R>
struct Velocity {
  R vx, vy, vz;
};

// Choose the process with u[1] against the cumulative rates and scatter
// (u[0] is unused: the candidate test drew from Philox2x32).
// Returns the new velocity; *proc_out = 0 elastic, 1 excitation,
// 2 ionization, 3 null (velocity unchanged).
template <typename R>
__device__ Velocity<R> collide(const InstDev& P, R kv, R vlim, R vx, R vy, R vz, R v1, R s1,
                               uint4 rr, uint32_t id, uint32_t step, R wj,
                               unsigned long long* acc, R* e_sec_out, int* proc_out) {
  const StepConsts<R>& K = consts<R>(P);
  R u[4];
  uniform4<R>(rr, u);
  atomicAdd(&acc[ACC_CAND], 1ull);
  R vb = v1 > vlim ? vlim : v1;
  if (vb > K.vb_cap) {
    vb = K.vb_cap;
    atomicAdd(&acc[ACC_MAJ], 1ull);
  }
  const R c = K.ndt * vb;
  const R eps = s1 * K.K_E;
  R xs[kMaxProc];
  xsec(P, eps, xs);
  const R rsel = u[1] * K.P0;
  // the first process whose cumulative rate exceeds the draw: elastic,
  // excitation level 1..n_exc, ionization; none: a null collision
  const int n_proc = P.n_exc + 2;
  int k = 0;
  while (k < n_proc && !(rsel < c * xs[k])) ++k;
  const int proc = k == n_proc ? 3 : (k == 0 ? 0 : (k <= P.n_exc ? 1 : 2));
  *proc_out = proc;
  Velocity<R> o = {vx, vy, vz};
  if (proc == 3) return o;
  atomicAdd(&acc[ACC_COLL0 + proc], 1ull);
  if (proc == 0) {
    // Vahedi-Surendra: cos chi = (2 + eps - 2 (1 + eps)^u) / eps, with
    // 1 - cos chi and 1 + cos chi each formed without cancellation so that
    // sin chi keeps its relative precision at both ends
    const R L = r_log1p(eps);
    const R em = r_expm1(u[2] * L);
    const R ep = -r_expm1(-((R)1 - u[2]) * L);
    R omc = (em + em) / eps;
    R opc = (((R)1 + eps) * (ep + ep)) / eps;
    omc = r_min((R)2, r_max((R)0, omc));
    opc = r_min((R)2, r_max((R)0, opc));
    const R cc = omc <= (R)1 ? (R)1 - omc : opc - (R)1;
    const R sc = r_sqrt(omc * opc);
    const R ph = K.two_pi * u[3];
    const R cp = r_cos(ph), sn = r_sin(ph);
    const R e_new = eps * ((R)1 - K.R2 * omc);
    R ux = vx / v1, uy = vy / v1, uz = vz / v1;
    rotate(ux, uy, uz, cc, sc, cp, sn);
    const R vn = r_sqrt(e_new * kv);
    o.vx = vn * ux;
    o.vy = vn * uy;
    o.vz = vn * uz;
  } else if (proc == 1) {
    R e_new = eps - K.e_ex[k - 1];
    if (e_new < (R)0) {
      e_new = (R)0;
      atomicAdd(&acc[ACC_CLAMP], 1ull);
    }
    isotropic(r_sqrt(e_new * kv), u[2], u[3], K.two_pi, o.vx, o.vy, o.vz);
  } else {
    R e_av = eps - K.e_io;
    if (e_av < (R)0) {
      e_av = (R)0;
      atomicAdd(&acc[ACC_CLAMP], 1ull);
    }
    atomicAdd(&acc[ACC_WIONZ], (unsigned long long)fixed_charge(wj, K.wscale));
    const uint4 r1 =
        philox4x32_10(make_uint4(id, step, P.ctr_inst * 2u, 1u), P.key0, P.key1);
    const R es = uniform01r<R>(r1.x) * e_av;
    const R ep = e_av - es;
    isotropic(r_sqrt(ep * kv), u[2], u[3], K.two_pi, o.vx, o.vy, o.vz);
    *e_sec_out = es;
  }
  return o;
}

// Write the electron and Ar+ born by an ionization at slots pe (electron
// store) and pi (ion store) with their serial numbers, and deposit both.  The
// secondary gets energy es along an isotropic direction (block 1 of the
// primary's draws); the ion a gas-temperature Maxwellian (Box-Muller on
// block 2).
template <typename R>
__device__ void born_pair(const InstDev& P, const SoAT<R>& me, const SoAT<R>& mi, uint32_t pe,
                          uint32_t pi, int cell, R off, R wj, uint32_t id, uint32_t step, R es,
                          uint32_t serial_e, uint32_t serial_i) {
  const StepConsts<R>& K = consts<R>(P);
  const uint32_t gen = id & kGenBit;
  const uint4 r1 = philox4x32_10(make_uint4(id, step, P.ctr_inst * 2u, 1u), P.key0, P.key1);
  R bx, by, bz;
  isotropic(r_sqrt(es * K.K_V[kElectron]), uniform01r<R>(r1.y), uniform01r<R>(r1.z), K.two_pi,
            bx, by, bz);
  me.cell[pe] = cell;
  me.off[pe] = off;
  me.vx[pe] = bx;
  me.vy[pe] = by;
  me.vz[pe] = bz;
  me.wj[pe] = wj;
  me.id[pe] = gen | (serial_e & kSerialMask);
  deposit(P.rho_acc[kElectron], cell, off,
          fixed_charge(beta_of(r_sqrt(bx * bx + by * by + bz * bz), K.vlim[kElectron]) * wj,
                       K.wscale));
  const uint4 r2 = philox4x32_10(make_uint4(id, step, P.ctr_inst * 2u, 2u), P.key0, P.key1);
  R g[4];
  uniform4<R>(r2, g);
  const R rr1 = r_sqrt((R)-2 * r_log(g[0]));
  const R rr2 = r_sqrt((R)-2 * r_log(g[2]));
  const R a1 = K.two_pi * g[1], a2 = K.two_pi * g[3];
  const R ix = K.sigT_ion * (rr1 * r_cos(a1));
  const R iy = K.sigT_ion * (rr1 * r_sin(a1));
  const R iz = K.sigT_ion * (rr2 * r_cos(a2));
  mi.cell[pi] = cell;
  mi.off[pi] = off;
  mi.vx[pi] = ix;
  mi.vy[pi] = iy;
  mi.vz[pi] = iz;
  mi.wj[pi] = wj;
  mi.id[pi] = gen | (serial_i & kSerialMask);
  deposit(P.rho_acc[kIon], cell, off,
          fixed_charge(beta_of(r_sqrt(ix * ix + iy * iy + iz * iz), K.vlim[kIon]) * wj,
                       K.wscale));
}

// Slot after the last live marker of a store (the particle kernel has
// compacted every tile of this step).
__device__ __forceinline__ uint32_t tail_slot(const SpeciesDev& S, const SpeciesState& st) {
  return st.n_tiles ? (st.n_tiles - 1) * (uint32_t)kTile + S.fill[st.cur][st.n_tiles - 1]
                    : 0u;
}

template <typename R>
__device__ __forceinline__ void write_marker(const SoAT<R>& d, size_t o, int cell, R off, R vx,
                                             R vy, R vz, R wj, uint32_t id) {
  d.cell[o] = cell;
  d.off[o] = off;
  d.vx[o] = vx;
  d.vy[o] = vy;
  d.vz[o] = vz;
  d.wj[o] = wj;
  d.id[o] = id;
}

}  // namespace

template <typename R>
__global__ void __launch_bounds__(kCollThreads) k_collide(DeviceRefs r) {
  __shared__ unsigned long long s_acc[ACC_COUNT];
  __shared__ uint32_t s_births[kCollWarps];
  __shared__ uint32_t s_prefix;
  __shared__ unsigned int s_chunk;
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
    R* esec = reinterpret_cast<R*>(E.esec);
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
    uint32_t warp_births = 0;
    if (!ion_chunk) {
      for (uint32_t c0 = 0; c0 < total; c0 += 32) {
        const uint32_t ce = c0 + lane;
        uint32_t q;
        const int j = locate_event(ce < total ? ce : total - 1, q);
        bool ionized = false;
        if (ce < total) {
          const size_t base = (size_t)(kw + j) * kTile;
          const uint32_t a = E.cand[base + q];
          const size_t o = base + a;
          const int cell = me.cell[o];
          const R off = me.off[o], wj = me.wj[o];
          const uint32_t id = me.id[o];
          R vx = me.vx[o], vy = me.vy[o], vz = me.vz[o];
          const R s1 = vx * vx + vy * vy + vz * vz;
          const R v1 = r_sqrt(s1);
          const uint4 rr =
              philox4x32_10(make_uint4(id, step, P.ctr_inst * 2u, 0u), P.key0, P.key1);
          int proc;
          R es = (R)0;
          const Velocity<R> nv =
              collide<R>(P, kv, vlim, vx, vy, vz, v1, s1, rr, id, step, wj, s_acc, &es, &proc);
          if (proc < 3) {
            vx = nv.vx;
            vy = nv.vy;
            vz = nv.vz;
            me.vx[o] = vx;
            me.vy[o] = vy;
            me.vz[o] = vz;
            if (proc == 2) {
              ionized = true;
              E.cand[base + q] = (uint16_t)(a | 0x8000u);  // mark for pass 2
              esec[base + q] = es;
            }
          }
          deposit(P.rho_acc[kElectron], cell, off,
                  fixed_charge(beta_of(r_sqrt(vx * vx + vy * vy + vz * vz), vlim) * wj,
                               K.wscale));
        }
        warp_births += __popc(__ballot_sync(0xFFFFFFFFu, ionized));
      }
    } else {
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
          const uint32_t a = ce < total ? E.cand[base + q] : 0u;
          const bool ionized = ce < total && (a & 0x8000u);
          const uint32_t b = __ballot_sync(0xFFFFFFFFu, ionized);
          if (ionized) {
            const uint32_t rank = off_w + ranked + __popc(b & lanemask_lt);
            const size_t o = base + (a & 0x7FFFu);
            const uint32_t pe = app_e + rank, pi = app_i + rank;
            if (pe >= cap_e || pi >= cap_i) {
              atomicCAS(&ctrl->error, 0, kErrCapacity);
            } else {
              born_pair<R>(P, me, mi, pe, pi, me.cell[o], me.off[o], me.wj[o], me.id[o], step,
                           esec[base + q], se.next_id + rank, si.next_id + rank);
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
  if (r.fp64) k_collide<double><<<grid, kCollThreads, 0, s>>>(r);
  else k_collide<float><<<grid, kCollThreads, 0, s>>>(r);
}

static_assert(kCollThreads == 32 * kCollWarps, "kCollWarps warps per chunk");
static_assert(kCollWarpTiles <= 32, "per-tile counts live one per lane");
static_assert(kTile <= 0x8000, "candidate slots leave the top bit for the ionization mark");

}  // namespace slpic
