// Host side of libslpic: the C ABI declared in include/slpic.h.  Validates
// and stores the configuration, derives the single-precision constants of
// the step, owns the device memory, and launches the step (directly or as a
// replayed CUDA graph of several steps).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <functional>
#include <limits>
#include <mutex>
#include <string>
#include <vector>

#include "slpic.h"
#include "slpic_internal.h"

using namespace slpic;

namespace {

// CODATA 2018 (SI).
const double kQe = 1.602176634e-19;
const double kKB = 1.380649e-23;
const double kEps0 = 8.8541878128e-12;
const double kTwoPi = 6.283185307179586;

constexpr int kGraphSteps = 32;  // steps captured in one CUDA graph
constexpr int kRingLen = 4096;   // per-step records kept on the device

std::string g_create_error;

struct HostSpecies {
  bool set = false;
  double mass = 0, charge = 0, vlim = 0;
  long long cap = 0;
};

struct HostInst {
  bool gap_set = false, gas_set = false, xs_set = false, dt_set = false;
  double d = 0, V = 0, area = 1;
  int n_cells = 0, field_mode = 0;
  double p_Pa = 0, T_K = 300;
  int lo_exp2 = 0, log2_sub = 0, octaves = 0;
  std::vector<float> el, io;
  int n_exc = 1;                  // excitation levels
  std::vector<float> ex[kMaxExc];  // their cross sections, in order
  double e_ex[kMaxExc] = {0, 0, 0};
  double e_io = 0;
  HostSpecies sp[2];
  double gamma = 0, dt = 0;
  int emission_model = 0;  // SLPIC_EMISSION_*
  int emit = 1;            // 0 while a breakdown search runs its avalanches
  uint64_t seed = 0;
  int shift = 32;
};

struct DevSpeciesAlloc {
  void* block = nullptr;
};

}  // namespace

struct slpic_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;
  int n_inst = 0;
  int fp64 = 0;  // marker path in double precision
  std::vector<HostInst> hi;
  std::string err;
  bool committed = false;
  // device memory
  std::vector<void*> allocs;
  InstDev* d_inst = nullptr;
  InstState* d_istate = nullptr;
  SpeciesState* d_sstate = nullptr;
  Control* d_ctrl = nullptr;
  unsigned int spin_limit = 0;  // bounded waits' polls (0: the default)
  Transfer* d_xfer = nullptr;
  unsigned int* d_seg = nullptr;
  unsigned int* d_scratch = nullptr;  // 16 bytes for small device results
  std::vector<InstDev> h_inst;  // host copies of the device configuration
  DeviceRefs refs{};
  int push_grid = 0;
  int move_grid = 0;
  int collide_grid = 0;
  int sms = 0;             // multiprocessors of the device
  int max_push_warps = 0;  // most particle-kernel warps per CTA that fit
  // shared-memory charge grid of the particle kernel (nodes of the largest
  // instance; 0: none fits) and the most warps that fit next to it; shapes
  // with more warps deposit to global memory
  int smem_nodes_full = 0;
  int max_push_warps_smem = 0;
  int collide_per_sm = 8;  // collision CTAs per SM
  int small_limit = kSmallMaxTiles;  // single-CTA path: most tiles per store (0: off)
  // per instance: stepped since its field was last reset (phi is then formed
  // from the last deposit when read)
  std::vector<char> stepped;
  // per instance with an imposed field: stepped since its last-step deposit
  // was formed (the step deposits nothing then; the deposit is formed from
  // the markers when read, or before they change)
  std::vector<char> dep_dirty;
  int blocks_per_sm = 0;
  // graph of kGraphSteps steps
  cudaGraphExec_t graph = nullptr;
  // profiling
  bool profiling = false;
  std::vector<cudaEvent_t> ev;  // pairs
  size_t ev_used = 0;
  double prof_ms = 0;
  long long prof_launches = 0;
  long long last_launches = 0;
};

namespace {

int fail(slpic_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else g_create_error = buf;
  return code;
}

int cuda_fail(slpic_ctx* c, cudaError_t e, const char* what) {
  return fail(c, SLPIC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                        \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

bool valid_inst(slpic_ctx* c, int inst) { return c && inst >= 0 && inst < c->n_inst; }

int set_device(slpic_ctx* c) {
  CK(cudaSetDevice(c->device), "cudaSetDevice");
  return SLPIC_OK;
}

int device_error(slpic_ctx* c) {
  Control h;
  CK(cudaMemcpy(&h, c->d_ctrl, sizeof h, cudaMemcpyDeviceToHost), "read status");
  switch (h.error) {
    case kErrNone: return SLPIC_OK;
    case kErrCapacity:
      return fail(c, SLPIC_ERR_CAPACITY,
                  "instance %d: live markers or births exceeded the capacity", h.error_inst);
    case kErrTimeout:
      return fail(c, SLPIC_ERR_TIMEOUT, "a bounded device wait timed out");
    case kErrIdWrap:
      return fail(c, SLPIC_ERR_CAPACITY, "instance %d: marker serial numbers exhausted (2^31)",
                  h.error_inst);
    default: return fail(c, SLPIC_ERR_CUDA, "unknown device error %d", h.error);
  }
}

int sync(slpic_ctx* c) {
  if (int rc = set_device(c)) return rc;
  CK(cudaStreamSynchronize(c->stream), "stream synchronize");
  if (!c->committed) return SLPIC_OK;
  return device_error(c);
}

// The step's constants in the marker path's type R, each rounded once from
// its double-precision definition; the majorant is formed in R from the R
// table, with the same operations the step uses.
template <typename R>
void derive_consts(const HostInst& h, StepConsts<R>& K) {
  const double dx = h.d / h.n_cells;
  const HostSpecies& E = h.sp[kElectron];
  const HostSpecies& I = h.sp[kIon];
  for (int s = 0; s < 2; ++s) {
    const HostSpecies& S = h.sp[s];
    const bool limited = S.vlim > 0.0 && std::isfinite(S.vlim);
    K.qmdt[s] = (R)((S.charge / S.mass) * h.dt);
    K.vlim[s] = limited ? (R)S.vlim : std::numeric_limits<R>::infinity();
    K.K_V[s] = (R)(2.0 * kQe / S.mass);
  }
  K.dtdx = (R)(h.dt / dx);
  K.K_E = (R)(0.5 * E.mass / kQe);
  const double n_g = h.p_Pa / (kKB * h.T_K);
  K.ndt = (R)(n_g * h.dt);
  K.R2 = (R)(2.0 * E.mass / I.mass);
  for (int k = 0; k < kMaxExc; ++k) K.e_ex[k] = (R)h.e_ex[k];
  K.e_io = (R)h.e_io;
  K.sigT_ion = (R)std::sqrt(kKB * h.T_K / I.mass);
  K.K_Ei = (R)(0.5 * I.mass / kQe);
  K.gamma = (R)h.gamma;
  K.wscale = (R)std::ldexp(1.0, h.shift);
  K.two_pi = (R)kTwoPi;
  K.e_lo = (R)std::ldexp(1.0, h.lo_exp2);
  K.e_hi = (R)std::ldexp(1.0, h.lo_exp2 + h.octaves);
  // majorant of n_g sigma_tot(eps) min(v, vlim) dt over the table
  R smax = 0;
  for (size_t j = 0; j < h.el.size(); ++j) {
    R s = (R)h.el[j];
    for (int k = 0; k < h.n_exc; ++k) s = s + (R)h.ex[k][j];
    s = s + (R)h.io[j];
    smax = std::max(smax, s);
  }
  const R v_top = std::sqrt(K.e_hi * K.K_V[kElectron]);
  K.vb_cap = std::min(K.vlim[kElectron], v_top);
  K.P0 = (K.ndt * K.vb_cap) * smax;
}

// Derive the constants of instance i (everything that does not need
// reallocation) into c->h_inst[i].
void fill_constants(slpic_ctx* c, int i, InstDev& P) {
  const HostInst& h = c->hi[i];
  const double dx = h.d / h.n_cells;
  P.n_cells = h.n_cells;
  P.field_mode = h.field_mode;
  P.charge_shift = h.shift;
  P.tab_lo_exp2 = h.lo_exp2;
  P.tab_log2_sub = h.log2_sub;
  P.tab_nodes = (h.octaves << h.log2_sub) + 1;
  P.n_exc = h.n_exc;
  P.key0 = (uint32_t)h.seed;
  P.key1 = (uint32_t)(h.seed >> 32);
  P.ctr_inst = (uint32_t)i;
  // key of the per-step null-collision draw: both seed words and the instance
  P.key2 = (uint32_t)h.seed ^ (uint32_t)(h.seed >> 32) ^ (0x85EBCA6Bu * (uint32_t)(i + 1));
  derive_consts(h, P.c32);
  derive_consts(h, P.c64);
  P.emission_model = h.emission_model;
  P.emit = h.emit;
  P.dx = dx;
  P.d = h.d;
  P.V = h.V;
  P.area = h.area;
  P.dt = h.dt;
  P.pois_C = kQe * dx * std::ldexp(1.0, -h.shift) / (h.area * kEps0);
}

int check_config(slpic_ctx* c, int i) {
  const HostInst& h = c->hi[i];
  if (!h.gap_set) return fail(c, SLPIC_ERR_STATE, "instance %d: slpic_set_gap not called", i);
  if (!h.gas_set) return fail(c, SLPIC_ERR_STATE, "instance %d: slpic_set_gas not called", i);
  if (!h.xs_set)
    return fail(c, SLPIC_ERR_STATE, "instance %d: slpic_set_cross_sections not called", i);
  if (!h.dt_set) return fail(c, SLPIC_ERR_STATE, "instance %d: slpic_set_dt not called", i);
  for (int s = 0; s < 2; ++s)
    if (!h.sp[s].set)
      return fail(c, SLPIC_ERR_STATE, "instance %d: species %d not configured", i, s);
  return SLPIC_OK;
}

template <typename T>
T* carve(char*& p, size_t n) {
  T* r = reinterpret_cast<T*>(p);
  p += (n * sizeof(T) + 255) & ~size_t(255);
  return r;
}

// Bytes of a store of n slots whose five real streams have rsz bytes each.
size_t soa_bytes(size_t n, size_t rsz) {
  return 2 * ((n * 4 + 255) & ~size_t(255)) + 5 * ((n * rsz + 255) & ~size_t(255));
}

SoA carve_soa(char*& p, size_t n, size_t rsz) {
  SoA s;
  s.cell = carve<int32_t>(p, n);
  s.off = reinterpret_cast<float*>(carve<char>(p, n * rsz));
  s.vx = reinterpret_cast<float*>(carve<char>(p, n * rsz));
  s.vy = reinterpret_cast<float*>(carve<char>(p, n * rsz));
  s.vz = reinterpret_cast<float*>(carve<char>(p, n * rsz));
  s.wj = reinterpret_cast<float*>(carve<char>(p, n * rsz));
  s.id = carve<uint32_t>(p, n);
  return s;
}

int dmalloc(slpic_ctx* c, void** p, size_t bytes, const char* what) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  c->allocs.push_back(*p);
  return SLPIC_OK;
}

// Reset the vacuum field of instance i on the device: phi linear, E = -V/d.
int reset_field(slpic_ctx* c, int i) {
  const InstDev& P = c->h_inst[i];
  const int nn = P.n_cells + 1;
  std::vector<double> phi(nn), E(nn, -P.V / P.d);
  std::vector<float> E32(nn, (float)(-P.V / P.d));
  for (int k = 0; k < nn; ++k) phi[k] = P.V * k / P.n_cells;
  CK(cudaMemcpyAsync(P.phi, phi.data(), nn * 8, cudaMemcpyHostToDevice, c->stream), "field");
  CK(cudaMemcpyAsync(P.E64, E.data(), nn * 8, cudaMemcpyHostToDevice, c->stream), "field");
  CK(cudaMemcpyAsync(P.E32, E32.data(), nn * 4, cudaMemcpyHostToDevice, c->stream), "field");
  CK(cudaStreamSynchronize(c->stream), "field");
  if ((int)c->stepped.size() == c->n_inst) c->stepped[i] = 0;
  return SLPIC_OK;
}

int upload_inst(slpic_ctx* c, int i) {
  CK(cudaMemcpyAsync(c->d_inst + i, &c->h_inst[i], sizeof(InstDev), cudaMemcpyHostToDevice,
                     c->stream),
     "upload instance");
  CK(cudaStreamSynchronize(c->stream), "upload instance");
  return SLPIC_OK;
}

int zero_counters(slpic_ctx* c, int i) {
  const InstDev& P = c->h_inst[i];
  CK(cudaMemsetAsync(P.acc, 0, ACC_COUNT * 8, c->stream), "reset");
  CK(cudaMemsetAsync(P.total, 0, sizeof(TallyRec), c->stream), "reset");
  CK(cudaMemsetAsync(P.ring, 0, sizeof(TallyRec) * P.ring_len, c->stream), "reset");
  // step counter, step count and seeded weight restart; the live weight
  // describes the markers, which stay
  InstState is;
  CK(cudaMemcpyAsync(&is, c->d_istate + i, sizeof is, cudaMemcpyDeviceToHost, c->stream), "reset");
  CK(cudaStreamSynchronize(c->stream), "reset");
  is.step = 0;
  is.n_steps_done = 0;
  is.w_seed = 0;
  is.ion_steps = 0;
  CK(cudaMemcpyAsync(c->d_istate + i, &is, sizeof is, cudaMemcpyHostToDevice, c->stream), "reset");
  for (int s = 0; s < 2; ++s) {
    CK(cudaMemsetAsync(P.rho_acc[s], 0, (P.n_cells + 1) * 8, c->stream), "reset");
    CK(cudaMemsetAsync(P.rho_last[s], 0, (P.n_cells + 1) * 8, c->stream), "reset");
  }
  if ((int)c->dep_dirty.size() == c->n_inst) c->dep_dirty[i] = 0;
  CK(cudaStreamSynchronize(c->stream), "reset");
  return SLPIC_OK;
}

int commit(slpic_ctx* c) {
  if (c->committed) return SLPIC_OK;
  for (int i = 0; i < c->n_inst; ++i)
    if (int rc = check_config(c, i)) return rc;
  if (int rc = set_device(c)) return rc;
  c->h_inst.assign(c->n_inst, InstDev{});
  int max_nodes = 0;
  unsigned long long total_tiles = 0;
  for (int i = 0; i < c->n_inst; ++i) {
    HostInst& h = c->hi[i];
    InstDev& P = c->h_inst[i];
    std::memset(&P, 0, sizeof P);
    fill_constants(c, i, P);
    const int nn = h.n_cells + 1;
    max_nodes = std::max(max_nodes, nn);
    // per-instance arrays
    const size_t tab_n = h.el.size() + 1;
    const int n_proc = h.n_exc + 2;
    const int stride = n_proc > 4 ? 2 : 1;  // float4s per node
    size_t bytes = 0;
    bytes += (tab_n * 16 * stride + 255) & ~size_t(255);
    if (c->fp64) bytes += (tab_n * sizeof(TabNode64) + 255) & ~size_t(255);
    bytes += ((nn * 4 + 255) & ~size_t(255));
    bytes += 2 * ((nn * 8 + 255) & ~size_t(255));
    bytes += 5 * ((nn * 8 + 255) & ~size_t(255)) + 256;
    bytes += 256 + ((sizeof(TallyRec) * kRingLen + 255) & ~size_t(255)) + 256;
    void* blk;
    if (int rc = dmalloc(c, &blk, bytes, "instance arrays")) return rc;
    char* p = (char*)blk;
    float4* tab = carve<float4>(p, tab_n * stride);
    P.table = tab;
    P.tab_stride = stride;
    TabNode64* tab64 = c->fp64 ? carve<TabNode64>(p, tab_n) : nullptr;
    P.table64 = tab64;
    P.E32 = carve<float>(p, nn);
    P.phi = carve<double>(p, nn);
    P.E64 = carve<double>(p, nn);
    P.rho_acc[0] = carve<unsigned long long>(p, nn);
    P.rho_acc[1] = carve<unsigned long long>(p, nn);
    P.rho_last[0] = carve<long long>(p, nn);
    P.rho_last[1] = carve<long long>(p, nn);
    P.pois_I = carve<long long>(p, nn);
    P.pois_D1 = carve<double>(p, 1);
    P.acc = carve<unsigned long long>(p, ACC_COUNT);
    P.ring = carve<TallyRec>(p, kRingLen);
    P.total = carve<TallyRec>(p, 1);
    P.ring_len = kRingLen;
    // cumulative tables: elastic, + each excitation level, + ionization, in
    // FP32 (and FP64) with one padding node equal to the last
    std::vector<float> hs((size_t)tab_n * 4 * stride, 0.0f);
    std::vector<TabNode64> hd(tab64 ? tab_n : 0);
    for (size_t j = 0; j + 1 < tab_n; ++j) {
      float sf = h.el[j];
      double sd = h.el[j];
      float* node = &hs[j * 4 * stride];
      node[0] = sf;
      if (tab64) hd[j].s[0] = sd;
      for (int k = 1; k < n_proc; ++k) {
        const float part = k <= h.n_exc ? h.ex[k - 1][j] : h.io[j];
        sf = sf + part;
        sd = sd + (double)part;
        node[k] = sf;
        if (tab64) hd[j].s[k] = sd;
      }
    }
    std::copy(hs.end() - 8 * stride, hs.end() - 4 * stride, hs.end() - 4 * stride);
    if (tab64) hd[tab_n - 1] = hd[tab_n - 2];
    CK(cudaMemcpy(tab, hs.data(), hs.size() * 4, cudaMemcpyHostToDevice), "table");
    if (tab64)
      CK(cudaMemcpy(tab64, hd.data(), tab_n * sizeof(TabNode64), cudaMemcpyHostToDevice),
         "table");
    // marker stores: tiles of kTile slots (two buffers for repacking);
    // electrons emitted at the cathode are staged in slots of the ion tile
    // that emitted them; collision candidates are queued per electron tile
    uint32_t cap_tiles[2];
    for (int s = 0; s < 2; ++s)
      cap_tiles[s] = (uint32_t)(((size_t)h.sp[s].cap + kTile - 1) / kTile + 1);
    for (int s = 0; s < 2; ++s) {
      SpeciesDev& S = P.sp[s];
      S.cap_tiles = cap_tiles[s];
      const size_t slots = (size_t)cap_tiles[s] * kTile;
      const size_t stage_b = s == kElectron ? (size_t)cap_tiles[kIon] * kTile : 0;
      const size_t cand_slots = s == kElectron ? slots : 0;
      const size_t arr = ((size_t)cap_tiles[s] + 1) * 4 + 256;
      const size_t rsz = c->fp64 ? 8 : 4;
      const size_t crsz = c->fp64 ? sizeof(CandRec<double>) : sizeof(CandRec<float>);
      size_t b = 2 * soa_bytes(slots, rsz) + soa_bytes(stage_b, rsz) + 4 * arr +
                 cand_slots * crsz + 512;
      void* sb;
      if (int rc = dmalloc(c, &sb, b, "marker buffers")) return rc;
      char* q = (char*)sb;
      S.buf[0] = carve_soa(q, slots, rsz);
      S.buf[1] = carve_soa(q, slots, rsz);
      if (stage_b) S.stage_b = carve_soa(q, stage_b, rsz);
      else std::memset(&S.stage_b, 0, sizeof(SoA));
      S.fill[0] = carve<uint32_t>(q, cap_tiles[s] + 1);
      S.fill[1] = carve<uint32_t>(q, cap_tiles[s] + 1);
      S.births = carve<uint32_t>(q, cap_tiles[s] + 1);
      S.n_cand = carve<uint32_t>(q, cap_tiles[s] + 1);
      S.crec = cand_slots ? (void*)carve<char>(q, cand_slots * crsz) : nullptr;
      CK(cudaMemset(S.fill[0], 0, ((size_t)cap_tiles[s] + 1) * 4), "fills");
      CK(cudaMemset(S.fill[1], 0, ((size_t)cap_tiles[s] + 1) * 4), "fills");
      total_tiles += cap_tiles[s];
    }
  }
  void* blk;
  const size_t nseg = 2 * (size_t)c->n_inst;
  // ordered-scan records: at most one chunk per kCollMinChunkTiles
  // (kMoveChunkTiles) tiles of every store, plus one partial chunk per store
  const size_t coll_chunks = total_tiles / kCollMinChunkTiles + nseg + 2;
  const size_t move_chunks = total_tiles / kMoveChunkTiles + nseg + 2;
  size_t bytes = ((sizeof(InstDev) * c->n_inst + 255) & ~size_t(255)) +
                 ((sizeof(InstState) * c->n_inst + 255) & ~size_t(255)) +
                 ((sizeof(SpeciesState) * nseg + 255) & ~size_t(255)) +
                 ((sizeof(Transfer) * nseg + 255) & ~size_t(255)) + 256 +
                 5 * ((4 * (nseg + 1) + 255) & ~size_t(255)) + 256 +
                 ((sizeof(ChunkStatus) * coll_chunks + 255) & ~size_t(255)) +
                 ((sizeof(ChunkStatus) * move_chunks + 255) & ~size_t(255));
  if (int rc = dmalloc(c, &blk, bytes, "control")) return rc;
  CK(cudaMemset(blk, 0, bytes), "control");
  char* p = (char*)blk;
  c->d_inst = carve<InstDev>(p, c->n_inst);
  c->d_istate = carve<InstState>(p, c->n_inst);
  c->d_sstate = carve<SpeciesState>(p, nseg);
  c->d_xfer = carve<Transfer>(p, nseg);
  c->d_ctrl = carve<Control>(p, 1);
  c->d_seg = carve<unsigned int>(p, nseg + 1);
  c->d_scratch = carve<unsigned int>(p, 4);
  c->refs.seg_wstart = carve<unsigned int>(p, nseg + 1);
  c->refs.coll_start = carve<unsigned int>(p, nseg + 1);
  c->refs.move_start = carve<unsigned int>(p, nseg + 1);
  c->refs.coll_tiles = carve<unsigned int>(p, nseg + 1);
  c->refs.coll_scan = carve<ChunkStatus>(p, coll_chunks);
  c->refs.move_scan = carve<ChunkStatus>(p, move_chunks);
  c->refs.inst = c->d_inst;
  c->refs.istate = c->d_istate;
  c->refs.sstate = c->d_sstate;
  c->refs.xfer = c->d_xfer;
  c->refs.ctrl = c->d_ctrl;
  CK(cudaMemcpy(&c->d_ctrl->spin_limit, &c->spin_limit, sizeof c->spin_limit,
                cudaMemcpyHostToDevice),
     "control");
  {
    // first step's electron collision chunks from the majorant probability:
    // about P0 kTile candidates per full tile
    std::vector<unsigned int> t(c->n_inst, (unsigned int)kCollMaxChunkTiles);
    for (int i = 0; i < c->n_inst; ++i) {
      const double P0 = c->fp64 ? c->h_inst[i].c64.P0 : (double)c->h_inst[i].c32.P0;
      const double per_tile = P0 * kTile;
      while (t[i] > (unsigned int)kCollMinChunkTiles &&
             t[i] / kCollWarps * per_tile > kCollTargetPerWarp)
        t[i] >>= 1;
    }
    CK(cudaMemcpy(c->refs.coll_tiles, t.data(), t.size() * 4, cudaMemcpyHostToDevice),
       "control");
  }
  c->refs.seg_start = c->d_seg;
  c->refs.n_inst = c->n_inst;
  // the whole charge grid of the largest instance goes to shared memory when
  // it fits next to the warps' marker stages (with at least 4 warps per CTA);
  // otherwise deposits use global atomics
  int smem_nodes = max_nodes <= 16385 ? max_nodes : 0;
  int bps = 0, warps = 0;
  size_t sbytes = 0;
  int e = push_config(c->fp64, smem_nodes, &warps, &bps, &sbytes);
  if (e != 0 || bps == 0) {
    smem_nodes = 0;
    e = push_config(c->fp64, 0, &warps, &bps, &sbytes);
    if (e != 0 || bps == 0) return fail(c, SLPIC_ERR_CUDA, "particle kernel cannot be launched");
  }
  c->refs.smem_nodes = smem_nodes;
  c->refs.push_warps = warps;
  c->refs.fp64 = c->fp64;
  c->smem_nodes_full = smem_nodes;
  c->max_push_warps_smem = smem_nodes ? warps : 0;
  int max_warps = warps;
  if (smem_nodes) {
    // more warps per CTA may fit when the deposits go to global memory
    int gw = 0, gbps = 0;
    size_t gbytes = 0;
    if (int e2 = push_config(c->fp64, 0, &gw, &gbps, &gbytes))
      return cuda_fail(c, (cudaError_t)e2, "particle kernel configuration");
    if (gbps > 0 && gw > warps) max_warps = gw;
  }
  {
    int net_nodes = 0;
    if (int e2 = finish_config(max_nodes, &net_nodes))
      return cuda_fail(c, (cudaError_t)e2, "finish kernel configuration");
    c->refs.finish_net_nodes = net_nodes;
  }
  if (int e2 = collide_config())
    return cuda_fail(c, (cudaError_t)e2, "collision kernel configuration");
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device), "attributes");
  c->sms = sms;
  c->max_push_warps = max_warps;
  c->blocks_per_sm = bps;
  c->push_grid = sms * bps;
  c->move_grid = sms * 2;
  c->collide_grid = sms * c->collide_per_sm;
  for (int i = 0; i < c->n_inst; ++i) {
    if (int rc = upload_inst(c, i)) return rc;
    if (int rc = reset_field(c, i)) return rc;
    if (int rc = zero_counters(c, i)) return rc;
  }
  CK(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking), "stream");
  c->committed = true;
  launch_finish(c->refs, 1, c->stream);
  CK(cudaGetLastError(), "plan");
  CK(cudaStreamSynchronize(c->stream), "plan");
  return SLPIC_OK;
}

int read_state(slpic_ctx* c, int inst, int sp, SpeciesState* out) {
  CK(cudaMemcpy(out, c->d_sstate + inst * 2 + sp, sizeof *out, cudaMemcpyDeviceToHost),
     "read state");
  return SLPIC_OK;
}

int write_state(slpic_ctx* c, int inst, int sp, const SpeciesState& st) {
  CK(cudaMemcpy(c->d_sstate + inst * 2 + sp, &st, sizeof st, cudaMemcpyHostToDevice),
     "write state");
  return SLPIC_OK;
}

// With an imposed field the step deposits nothing: form the last step's
// deposit of instance i from its markers (a function of them) if it has
// stepped since the deposit was last formed.  Called before the deposit is
// read and before the markers change.
int materialize_deposit(slpic_ctx* c, int i) {
  if (c->h_inst[i].field_mode == 1 || !c->dep_dirty[i]) return SLPIC_OK;
  SpeciesState st[2];
  CK(cudaMemcpyAsync(st, c->d_sstate + 2 * i, sizeof st, cudaMemcpyDeviceToHost, c->stream),
     "deposit");
  CK(cudaStreamSynchronize(c->stream), "deposit");
  const InstDev& P = c->h_inst[i];
  for (int s = 0; s < 2; ++s)
    CK(cudaMemsetAsync(P.rho_last[s], 0, (P.n_cells + 1) * 8, c->stream), "deposit");
  launch_deposit(c->refs, i, (int)(st[0].n_tiles + st[1].n_tiles), c->stream);
  CK(cudaGetLastError(), "deposit");
  c->dep_dirty[i] = 0;
  return SLPIC_OK;
}

void mark_stepped(slpic_ctx* c) {
  std::fill(c->stepped.begin(), c->stepped.end(), 1);
  for (int i = 0; i < c->n_inst; ++i)
    if (c->h_inst[i].field_mode != 1) c->dep_dirty[i] = 1;
}

int replan(slpic_ctx* c) {
  launch_finish(c->refs, 1, c->stream);
  CK(cudaGetLastError(), "plan");
  return SLPIC_OK;
}

int prepare(slpic_ctx* c) {
  if (int rc = commit(c)) return rc;
  if (int rc = set_device(c)) return rc;
  return SLPIC_OK;
}

// Single-CTA path (small.cu): up to n steps while every store has at most
// c->small_limit tiles; synchronous.  *done = steps run (0 when the path does
// not apply now).  It applies when every store is that small, every store
// can take the births of one step from there (so no capacity error can occur
// in it), the field-mode-1 grids fit in shared memory, and all instances fit
// on the device at once.  extra_ok (may be NULL) adds a condition per
// instance on its live counts.
int run_small(slpic_ctx* c, int64_t n, int64_t* done,
              const std::function<bool(int, int64_t, int64_t)>& extra_ok = nullptr) {
  *done = 0;
  if (n <= 0 || c->small_limit <= 0 || c->profiling) return SLPIC_OK;
  if (int rc = sync(c)) return rc;
  std::vector<SpeciesState> st(2 * (size_t)c->n_inst);
  CK(cudaMemcpy(st.data(), c->d_sstate, sizeof(SpeciesState) * st.size(),
                cudaMemcpyDeviceToHost),
     "small path");
  const int64_t L = (int64_t)c->small_limit * kTile;
  int max_pn = 0;
  for (int i = 0; i < c->n_inst; ++i) {
    const SpeciesState &e = st[2 * i], &o = st[2 * i + 1];
    if ((int)e.n_tiles > c->small_limit || (int)o.n_tiles > c->small_limit) return SLPIC_OK;
    if (c->hi[i].sp[kElectron].cap < 3 * L || c->hi[i].sp[kIon].cap < 2 * L) return SLPIC_OK;
    if (extra_ok && !extra_ok(i, e.n_live, o.n_live)) return SLPIC_OK;
    if (c->h_inst[i].field_mode == 1) max_pn = std::max(max_pn, c->h_inst[i].n_cells + 1);
  }
  size_t smem = 0;
  int bps = 0;
  if (int e = small_config(c->fp64, max_pn, &smem, &bps))
    return cuda_fail(c, (cudaError_t)e, "small path configuration");
  if (bps == 0 || (c->n_inst > 1 && (int64_t)bps * c->sms < c->n_inst)) return SLPIC_OK;
  // the grid barrier counts arrivals in 32 bits: launches of at most 2^30
  // arrivals (steps x instances), one after another
  const int64_t per_launch = std::max<int64_t>(1, (int64_t(1) << 30) / c->n_inst);
  const size_t off0 = offsetof(Control, small_bar);
  c->last_launches = 0;
  while (*done < n) {
    const int64_t k = std::min(n - *done, per_launch);
    CK(cudaMemsetAsync((char*)c->d_ctrl + off0, 0, offsetof(Control, small_done) + 8 - off0,
                       c->stream),
       "small path");
    if (int e = launch_small(c->refs, k, c->small_limit, smem, c->stream))
      return cuda_fail(c, (cudaError_t)e, "small path launch");
    launch_finish(c->refs, 1, c->stream);  // the batched path's next step
    CK(cudaGetLastError(), "small path");
    CK(cudaStreamSynchronize(c->stream), "small path");
    long long d = 0;
    CK(cudaMemcpy(&d, &c->d_ctrl->small_done, sizeof d, cudaMemcpyDeviceToHost),
       "small path");
    *done += d;
    c->last_launches += 2;
    if (d > 0) mark_stepped(c);
    if (int rc = device_error(c)) return rc;
    if (d < k) break;  // a store outgrew the path
  }
  return SLPIC_OK;
}

void drop_graph(slpic_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
}

int build_graph(slpic_ctx* c) {
  if (c->graph) return SLPIC_OK;
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal), "capture");
  for (int k = 0; k < kGraphSteps; ++k) {
    launch_push(c->refs, c->push_grid, c->capture_stream);
    launch_collide(c->refs, c->collide_grid, c->capture_stream);
    launch_finish(c->refs, 0, c->capture_stream);
    launch_move(c->refs, c->move_grid, c->capture_stream);
  }
  CK(cudaStreamEndCapture(c->capture_stream, &g), "capture");
  cudaError_t e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->graph = nullptr;
    return cuda_fail(c, e, "graph instantiate");
  }
  return SLPIC_OK;
}

// Launch shape of the step: warps per particle-kernel CTA (the super-tile
// size, so the next step is replanned) and collision CTAs per SM.  Results do
// not depend on it: tiles are independent, deposits are integer sums and
// births are ordered by (tile, slot).
int apply_shape(slpic_ctx* c, int warps, int coll_per_sm) {
  if (warps < 4 || warps > c->max_push_warps || warps % 4 || coll_per_sm < 1 || coll_per_sm > 32)
    return fail(c, SLPIC_ERR_INVALID_ARG,
                "launch shape: push warps must be a multiple of 4 in [4, %d], collision CTAs "
                "per SM in [1, 32]",
                c->max_push_warps);
  // the shared charge grid while it fits next to the warps' stages, else
  // deposits to global memory (the same integers either way)
  const int nodes = warps <= c->max_push_warps_smem ? c->smem_nodes_full : 0;
  int bps = 0;
  if (int e = push_blocks_per_sm(c->fp64, warps, nodes, &bps))
    return cuda_fail(c, (cudaError_t)e, "launch shape");
  if (bps < 1) return fail(c, SLPIC_ERR_CUDA, "launch shape: particle kernel does not fit");
  if (int rc = sync(c)) return rc;
  drop_graph(c);
  c->refs.smem_nodes = nodes;
  c->refs.push_warps = warps;
  c->blocks_per_sm = bps;
  c->push_grid = c->sms * bps;
  c->collide_per_sm = coll_per_sm;
  c->collide_grid = c->sms * coll_per_sm;
  if (int rc = replan(c)) return rc;
  return sync(c);
}

// The seven marker arrays of a caller (cell, off, vx, vy, vz, w_j, id), in
// the precision the call names.
struct Arrays {
  void* f[7];
  int fp64;
};

Arrays arrays_of(const slpic_soa_f32* s) {
  Arrays a{};
  if (s) {
    void* f[7] = {s->cell, s->off, s->vx, s->vy, s->vz, s->wj, s->id};
    std::memcpy(a.f, f, sizeof f);
  }
  a.fp64 = 0;
  return a;
}

Arrays arrays_of(const slpic_soa_f64* s) {
  Arrays a{};
  if (s) {
    void* f[7] = {s->cell, s->off, s->vx, s->vy, s->vz, s->wj, s->id};
    std::memcpy(a.f, f, sizeof f);
  }
  a.fp64 = 1;
  return a;
}

int arrays_check(slpic_ctx* c, const Arrays& a) {
  for (int k = 0; k < 7; ++k)
    if (!a.f[k]) return fail(c, SLPIC_ERR_INVALID_ARG, "null marker array");
  return SLPIC_OK;
}

int precision_check(slpic_ctx* c, int fp64) {
  if (fp64 != c->fp64)
    return fail(c, SLPIC_ERR_STATE,
                "the context's marker path is FP%d: use the %s marker calls", c->fp64 ? 64 : 32,
                c->fp64 ? "_f64" : "FP32");
  return SLPIC_OK;
}

// Bytes of field k of n markers.
size_t field_bytes(const slpic_ctx* c, int k, size_t n) {
  return (k == 0 || k == 6) ? n * 4 : n * (c->fp64 ? 8 : 4);
}

}  // namespace

extern "C" {

int slpic_version(void) { return 100; }

const char* slpic_last_error(const slpic_ctx* c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

int philox_static_setup_for(int device);

int slpic_create(slpic_ctx** out, int device, int n_instances) {
  if (!out) return fail(nullptr, SLPIC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_instances < 1 || n_instances > (1 << 20))
    return fail(nullptr, SLPIC_ERR_INVALID_ARG, "n_instances must be in [1, 2^20]");
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return fail(nullptr, SLPIC_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
  if (device < 0 || device >= n) return fail(nullptr, SLPIC_ERR_INVALID_ARG, "bad device %d", device);
  // slpic_philox_static's set-up for this device now, while memory is free
  // and before any stream capture (the caller's current device is kept)
  if (int rc = philox_static_setup_for(device)) return rc;
  slpic_ctx* c = new slpic_ctx;
  c->device = device;
  c->n_inst = n_instances;
  c->hi.resize(n_instances);
  c->stepped.assign(n_instances, 0);
  c->dep_dirty.assign(n_instances, 0);
  *out = c;
  return SLPIC_OK;
}

int slpic_destroy(slpic_ctx* c) {
  if (!c) return SLPIC_OK;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graph(c);
  for (auto& e : c->ev) cudaEventDestroy(e);
  for (void* p : c->allocs) cudaFree(p);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  delete c;
  return SLPIC_OK;
}

int slpic_set_stream(slpic_ctx* c, void* stream) {
  if (!c) return SLPIC_ERR_INVALID_ARG;
  c->stream = (cudaStream_t)stream;
  return SLPIC_OK;
}

int slpic_set_gap(slpic_ctx* c, int inst, double d, int n_cells, double V, int field_mode,
                  double area) {
  if (!valid_inst(c, inst)) return fail(c, SLPIC_ERR_INVALID_ARG, "bad instance");
  if (!(d > 0) || n_cells < 2 || n_cells > (1 << 24) || !std::isfinite(V) ||
      (field_mode != SLPIC_FIELD_FROZEN && field_mode != SLPIC_FIELD_POISSON) || !(area > 0))
    return fail(c, SLPIC_ERR_INVALID_ARG, "bad gap parameters");
  HostInst& h = c->hi[inst];
  if (c->committed && (n_cells != h.n_cells))
    return fail(c, SLPIC_ERR_STATE, "the cell count cannot change after the first use");
  h.d = d;
  h.n_cells = n_cells;
  h.V = V;
  h.field_mode = field_mode;
  h.area = area;
  h.gap_set = true;
  if (c->committed) {
    fill_constants(c, inst, c->h_inst[inst]);
    if (int rc = upload_inst(c, inst)) return rc;
    return reset_field(c, inst);
  }
  return SLPIC_OK;
}

int slpic_set_voltage(slpic_ctx* c, int inst, double V) {
  if (!valid_inst(c, inst) || !std::isfinite(V)) return fail(c, SLPIC_ERR_INVALID_ARG, "bad voltage");
  HostInst& h = c->hi[inst];
  if (!h.gap_set) return fail(c, SLPIC_ERR_STATE, "slpic_set_gap first");
  return slpic_set_gap(c, inst, h.d, h.n_cells, V, h.field_mode, h.area);
}

int slpic_set_gas(slpic_ctx* c, int inst, double p_Pa, double T_K) {
  if (!valid_inst(c, inst)) return fail(c, SLPIC_ERR_INVALID_ARG, "bad instance");
  if (!(p_Pa >= 0) || !std::isfinite(p_Pa) || !(T_K > 0))
    return fail(c, SLPIC_ERR_INVALID_ARG, "bad gas parameters");
  c->hi[inst].p_Pa = p_Pa;
  c->hi[inst].T_K = T_K;
  c->hi[inst].gas_set = true;
  if (c->committed) {
    fill_constants(c, inst, c->h_inst[inst]);
    return upload_inst(c, inst);
  }
  return SLPIC_OK;
}

int slpic_set_cross_sections_levels(slpic_ctx* c, int inst, int lo_exp2, int log2_sub,
                                    int octaves, const float* el, int n_exc,
                                    const float* const* ex, const double* e_ex,
                                    const float* io, double e_io) {
  if (!c) return SLPIC_ERR_INVALID_ARG;
  if (inst < -1 || inst >= c->n_inst) return fail(c, SLPIC_ERR_INVALID_ARG, "bad instance");
  if (n_exc < 1 || n_exc > kMaxExc || !ex || !e_ex)
    return fail(c, SLPIC_ERR_INVALID_ARG, "n_exc must be in [1, %d]", kMaxExc);
  if (!el || !io || log2_sub < 0 || log2_sub > 16 || octaves < 1 || octaves > 64 ||
      lo_exp2 < -100 || lo_exp2 + octaves > 100 || !(e_io >= 0))
    return fail(c, SLPIC_ERR_INVALID_ARG, "bad cross-section table");
  for (int k = 0; k < n_exc; ++k)
    if (!ex[k] || !(e_ex[k] >= 0))
      return fail(c, SLPIC_ERR_INVALID_ARG, "bad excitation level %d", k);
  const size_t n = ((size_t)octaves << log2_sub) + 1;
  auto ok = [](float v) { return v >= 0 && std::isfinite(v); };
  for (size_t j = 0; j < n; ++j) {
    bool good = ok(el[j]) && ok(io[j]);
    for (int k = 0; k < n_exc; ++k) good = good && ok(ex[k][j]);
    if (!good) return fail(c, SLPIC_ERR_INVALID_ARG, "cross sections must be finite and >= 0");
  }
  if (c->committed) return fail(c, SLPIC_ERR_STATE, "tables cannot change after the first use");
  const int lo = inst < 0 ? 0 : inst, hi = inst < 0 ? c->n_inst : inst + 1;
  for (int i = lo; i < hi; ++i) {
    HostInst& h = c->hi[i];
    h.lo_exp2 = lo_exp2;
    h.log2_sub = log2_sub;
    h.octaves = octaves;
    h.el.assign(el, el + n);
    h.n_exc = n_exc;
    for (int k = 0; k < kMaxExc; ++k) {
      if (k < n_exc) {
        h.ex[k].assign(ex[k], ex[k] + n);
        h.e_ex[k] = e_ex[k];
      } else {
        h.ex[k].clear();
        h.e_ex[k] = 0;
      }
    }
    h.io.assign(io, io + n);
    h.e_io = e_io;
    h.xs_set = true;
  }
  return SLPIC_OK;
}

int slpic_set_cross_sections(slpic_ctx* c, int inst, int lo_exp2, int log2_sub, int octaves,
                             const float* el, const float* ex, double e_ex, const float* io,
                             double e_io) {
  if (!ex) return fail(c, SLPIC_ERR_INVALID_ARG, "bad cross-section table");
  const float* levels[1] = {ex};
  const double th[1] = {e_ex};
  return slpic_set_cross_sections_levels(c, inst, lo_exp2, log2_sub, octaves, el, 1, levels, th,
                                         io, e_io);
}

int slpic_set_species(slpic_ctx* c, int inst, int species, double mass, double charge,
                      double v_lim, int64_t capacity) {
  if (!valid_inst(c, inst) || (species != 0 && species != 1))
    return fail(c, SLPIC_ERR_INVALID_ARG, "bad instance or species");
  if (!(mass > 0) || !std::isfinite(charge) || std::isnan(v_lim) || capacity < 1 ||
      capacity > (int64_t)0x7FFFFFFF - kTile)
    return fail(c, SLPIC_ERR_INVALID_ARG, "bad species parameters");
  HostSpecies& S = c->hi[inst].sp[species];
  if (c->committed && capacity != S.cap)
    return fail(c, SLPIC_ERR_STATE, "capacity cannot change after the first use");
  S.mass = mass;
  S.charge = charge;
  S.vlim = v_lim;
  S.cap = capacity;
  S.set = true;
  if (c->committed) {
    fill_constants(c, inst, c->h_inst[inst]);
    return upload_inst(c, inst);
  }
  return SLPIC_OK;
}

int slpic_set_emission(slpic_ctx* c, int inst, double g) {
  if (!valid_inst(c, inst) || !(g >= 0 && g <= 1)) return fail(c, SLPIC_ERR_INVALID_ARG, "gamma must be in [0, 1]");
  c->hi[inst].gamma = g;
  if (c->committed) {
    fill_constants(c, inst, c->h_inst[inst]);
    return upload_inst(c, inst);
  }
  return SLPIC_OK;
}

namespace {

// Re-derive and upload the constants of a committed instance.
int refresh_inst(slpic_ctx* c, int inst) {
  if (!c->committed) return SLPIC_OK;
  fill_constants(c, inst, c->h_inst[inst]);
  return upload_inst(c, inst);
}

}  // namespace

int slpic_set_emission_model(slpic_ctx* c, int inst, int model) {
  if (!valid_inst(c, inst) ||
      (model != SLPIC_EMISSION_CONSTANT && model != SLPIC_EMISSION_ENERGY))
    return fail(c, SLPIC_ERR_INVALID_ARG, "bad emission model");
  c->hi[inst].emission_model = model;
  return refresh_inst(c, inst);
}

int slpic_set_dt(slpic_ctx* c, int inst, double dt) {
  if (!valid_inst(c, inst) || !(dt >= 0) || !std::isfinite(dt))
    return fail(c, SLPIC_ERR_INVALID_ARG, "dt must be finite and >= 0");
  c->hi[inst].dt = dt;
  c->hi[inst].dt_set = true;
  if (c->committed) {
    fill_constants(c, inst, c->h_inst[inst]);
    return upload_inst(c, inst);
  }
  return SLPIC_OK;
}

int slpic_set_seed(slpic_ctx* c, int inst, uint64_t seed) {
  if (!valid_inst(c, inst)) return fail(c, SLPIC_ERR_INVALID_ARG, "bad instance");
  c->hi[inst].seed = seed;
  if (c->committed) {
    fill_constants(c, inst, c->h_inst[inst]);
    return upload_inst(c, inst);
  }
  return SLPIC_OK;
}

int slpic_set_charge_shift(slpic_ctx* c, int inst, int shift) {
  if (!valid_inst(c, inst) || shift < 0 || shift > 40)
    return fail(c, SLPIC_ERR_INVALID_ARG, "shift must be in [0, 40]");
  if (c->committed) return fail(c, SLPIC_ERR_STATE, "shift cannot change after the first use");
  c->hi[inst].shift = shift;
  return SLPIC_OK;
}

int slpic_suggest_dt(double d, int n_cells, double V, double m_ion, int mode, double* dt) {
  if (!dt || !(d > 0) || n_cells < 1 || !(V > 0) || !(m_ion > 0) || (mode != 0 && mode != 1))
    return SLPIC_ERR_INVALID_ARG;
  const double me = 9.1093837015e-31;
  const double m = mode == 0 ? m_ion : me;
  *dt = (d / n_cells) / std::sqrt(2.0 * kQe * V / m);
  return SLPIC_OK;
}

}  // extern "C"

namespace {

// Set the fills of tiles [first, ceil(end / kTile)) of a store whose slots
// [first * kTile, end) are all live.
int write_fills(slpic_ctx* c, const SpeciesDev& S, uint32_t cur, uint32_t first, uint32_t end) {
  const uint32_t last = (end + kTile - 1) / kTile;
  if (last <= first) return SLPIC_OK;
  std::vector<uint32_t> f(last - first);
  for (uint32_t k = first; k < last; ++k)
    f[k - first] = std::min<uint32_t>(end - k * (uint32_t)kTile, (uint32_t)kTile);
  CK(cudaMemcpy(S.fill[cur] + first, f.data(), f.size() * 4, cudaMemcpyHostToDevice), "fills");
  return SLPIC_OK;
}

// First free slot after the last live marker of a store.
int tail_slot(slpic_ctx* c, const SpeciesDev& S, const SpeciesState& st, uint32_t* out) {
  if (st.n_tiles == 0) {
    *out = 0;
    return SLPIC_OK;
  }
  uint32_t f = 0;
  CK(cudaMemcpy(&f, S.fill[st.cur] + st.n_tiles - 1, 4, cudaMemcpyDeviceToHost), "fills");
  *out = (st.n_tiles - 1) * (uint32_t)kTile + f;
  return SLPIC_OK;
}

}  // namespace

extern "C" int slpic_seed(slpic_ctx* c, int inst, int species, int64_t n, int mode, double e0,
                          double e_lo, double e_hi, double wj) {
  if (!valid_inst(c, inst) || (species != 0 && species != 1) || n < 0 || mode < 0 || mode > 3)
    return fail(c, SLPIC_ERR_INVALID_ARG, "bad seed arguments");
  if (!(wj >= 0) || !std::isfinite(wj) || !(e0 >= 0) || (mode == 2 && !(e_lo > 0 && e_hi >= e_lo)))
    return fail(c, SLPIC_ERR_INVALID_ARG, "bad seed energies or weight");
  if (int rc = prepare(c)) return rc;
  if (int rc = sync(c)) return rc;
  if (int rc = materialize_deposit(c, inst)) return rc;
  SpeciesState st;
  if (int rc = read_state(c, inst, species, &st)) return rc;
  const InstDev& P = c->h_inst[inst];
  const SpeciesDev& S = P.sp[species];
  uint32_t app = 0;
  if (int rc = tail_slot(c, S, st, &app)) return rc;
  if ((uint64_t)app + (uint64_t)n > (uint64_t)S.cap_tiles * kTile)
    return fail(c, SLPIC_ERR_CAPACITY, "seeding %lld markers exceeds the capacity", (long long)n);
  if ((uint64_t)st.next_id + (uint64_t)n > kSerialMask)
    return fail(c, SLPIC_ERR_CAPACITY, "marker serial numbers exhausted");
  // the weight in the marker path's type, and its fixed-point charge
  const double wr = c->fp64 ? wj : (double)(float)wj;
  const double wq = wr * P.c64.wscale;  // exact: a power-of-two scaling
  if (!(wq < 549755813888.0))
    return fail(c, SLPIC_ERR_INVALID_ARG,
                "weight %g is too large for charge shift %d (w 2^shift must stay below 2^39)", wj,
                P.charge_shift);
  const HostInst& h = c->hi[inst];
  // each parameter is rounded once to the marker path's type on the device
  const double ekin = mode == 3 ? std::sqrt(kKB * h.T_K / h.sp[species].mass) : e0;
  const double lr = mode == 2 ? std::log(e_hi / e_lo) : 0.0;
  launch_seed(c->refs, inst, species, app, st.next_id, (uint32_t)n, mode, ekin, e_lo, lr, wj,
              c->stream);
  CK(cudaGetLastError(), "seed");
  CK(cudaStreamSynchronize(c->stream), "seed");
  if (int rc = write_fills(c, S, st.cur, app / kTile, app + (uint32_t)n)) return rc;
  st.n_live += (uint32_t)n;
  st.next_id += (uint32_t)n;
  st.n_tiles = std::max(st.n_tiles, (app + (uint32_t)n + kTile - 1) / (uint32_t)kTile);
  if (int rc = write_state(c, inst, species, st)) return rc;
  {
    InstState is;
    CK(cudaMemcpy(&is, c->d_istate + inst, sizeof is, cudaMemcpyDeviceToHost), "seed");
    const unsigned long long q = (unsigned long long)n * (unsigned long long)std::llrint(wq);
    if (species == kElectron) is.w_seed += q;
    is.w_live[species] += q;
    CK(cudaMemcpy(c->d_istate + inst, &is, sizeof is, cudaMemcpyHostToDevice), "seed");
  }
  if (int rc = replan(c)) return rc;
  return sync(c);
}

namespace {

int load_common(slpic_ctx* c, int inst, int species, const Arrays& src, int64_t n,
                uint32_t next_id, cudaMemcpyKind kind) {
  if (!valid_inst(c, inst) || (species != 0 && species != 1) || n < 0)
    return fail(c, SLPIC_ERR_INVALID_ARG, "bad load arguments");
  if (int rc = precision_check(c, src.fp64)) return rc;
  if (n > 0)
    if (int rc = arrays_check(c, src)) return rc;
  if (next_id > kSerialMask) return fail(c, SLPIC_ERR_INVALID_ARG, "next_id beyond 2^31 - 1");
  if (int rc = prepare(c)) return rc;
  if (int rc = sync(c)) return rc;
  if (int rc = materialize_deposit(c, inst)) return rc;
  const InstDev& P = c->h_inst[inst];
  const SpeciesDev& S = P.sp[species];
  if ((uint64_t)n > (uint64_t)S.cap_tiles * kTile)
    return fail(c, SLPIC_ERR_CAPACITY, "%lld markers exceed the capacity", (long long)n);
  SpeciesState st;
  if (int rc = read_state(c, inst, species, &st)) return rc;
  const SoA& d = S.buf[st.cur];
  if (n > 0) {
    void* dst[7] = {d.cell, d.off, d.vx, d.vy, d.vz, d.wj, d.id};
    for (int k = 0; k < 7; ++k)
      CK(cudaMemcpyAsync(dst[k], src.f[k], field_bytes(c, k, (size_t)n), kind, c->stream),
         "load");
  }
  // validate on the device: a marker outside the gap would make the step
  // read and write outside the field and charge arrays
  unsigned int* scratch = c->d_scratch;
  unsigned int bad_init[4] = {0xFFFFFFFFu, 0u, 0u, 0u};
  CK(cudaMemcpyAsync(scratch, bad_init, 16, cudaMemcpyHostToDevice, c->stream), "load");
  launch_validate(c->fp64, d, (uint32_t)n, P.n_cells, P.charge_shift, scratch,
                  reinterpret_cast<unsigned long long*>(scratch + 2), c->stream);
  CK(cudaGetLastError(), "validate");
  unsigned int res[4];
  CK(cudaMemcpyAsync(res, scratch, 16, cudaMemcpyDeviceToHost, c->stream), "load");
  CK(cudaStreamSynchronize(c->stream), "load");
  st.n_live = 0;
  st.n_tiles = 0;
  if (res[0] != 0xFFFFFFFFu) {
    write_state(c, inst, species, st);
    replan(c);
    return fail(c, SLPIC_ERR_INVALID_ARG,
                "marker %u outside the gap, not finite, or with a weight of 2^39 charge "
                "units or more; the species was emptied", res[0]);
  }
  if (int rc = write_fills(c, S, st.cur, 0, (uint32_t)n)) return rc;
  st.n_live = (uint32_t)n;
  st.n_tiles = (uint32_t)(((uint64_t)n + kTile - 1) / kTile);
  st.next_id = next_id;
  if (int rc = write_state(c, inst, species, st)) return rc;
  {
    InstState is;
    CK(cudaMemcpy(&is, c->d_istate + inst, sizeof is, cudaMemcpyDeviceToHost), "load");
    unsigned long long wsum;
    std::memcpy(&wsum, res + 2, 8);
    if (species == kElectron) is.w_seed = wsum;
    is.w_live[species] = wsum;
    CK(cudaMemcpy(c->d_istate + inst, &is, sizeof is, cudaMemcpyHostToDevice), "load");
  }
  if (int rc = replan(c)) return rc;
  return sync(c);
}

}  // namespace

extern "C" {

int slpic_load_particles(slpic_ctx* c, int inst, int species, const slpic_soa_f32* host,
                         int64_t n, uint32_t next_id) {
  return load_common(c, inst, species, arrays_of(host), n, next_id, cudaMemcpyHostToDevice);
}

int slpic_load_particles_device(slpic_ctx* c, int inst, int species, const slpic_soa_f32* dev,
                                int64_t n, uint32_t next_id) {
  return load_common(c, inst, species, arrays_of(dev), n, next_id, cudaMemcpyDeviceToDevice);
}

int slpic_load_particles_f64(slpic_ctx* c, int inst, int species, const slpic_soa_f64* host,
                             int64_t n, uint32_t next_id) {
  return load_common(c, inst, species, arrays_of(host), n, next_id, cudaMemcpyHostToDevice);
}

int slpic_set_precision(slpic_ctx* c, int bits) {
  if (!c || (bits != 32 && bits != 64))
    return fail(c, SLPIC_ERR_INVALID_ARG, "precision must be 32 or 64");
  if (c->committed && (bits == 64) != (c->fp64 != 0))
    return fail(c, SLPIC_ERR_STATE, "the precision cannot change after the first use");
  c->fp64 = bits == 64 ? 1 : 0;
  return SLPIC_OK;
}

int slpic_reset_counters(slpic_ctx* c, int inst) {
  if (!valid_inst(c, inst)) return fail(c, SLPIC_ERR_INVALID_ARG, "bad instance");
  if (int rc = prepare(c)) return rc;
  if (int rc = sync(c)) return rc;
  return zero_counters(c, inst);
}

int slpic_step(slpic_ctx* c, int64_t n) {
  if (!c || n < 0) return fail(c, SLPIC_ERR_INVALID_ARG, "bad step count");
  if (int rc = prepare(c)) return rc;
  if (n > 0) mark_stepped(c);
  c->last_launches = 0;
  if (c->profiling) {
    for (int64_t k = 0; k < n; ++k) {
      if (c->ev_used + 2 > c->ev.size()) {
        for (int j = 0; j < 64; ++j) {
          cudaEvent_t e;
          CK(cudaEventCreate(&e), "event");
          c->ev.push_back(e);
        }
      }
      cudaEvent_t a = c->ev[c->ev_used], b = c->ev[c->ev_used + 1];
      c->ev_used += 2;
      CK(cudaEventRecord(a, c->stream), "event");
      launch_push(c->refs, c->push_grid, c->stream);
      CK(cudaEventRecord(b, c->stream), "event");
      launch_collide(c->refs, c->collide_grid, c->stream);
      launch_finish(c->refs, 0, c->stream);
      launch_move(c->refs, c->move_grid, c->stream);
      c->last_launches += 4;
    }
    CK(cudaGetLastError(), "step");
    return SLPIC_OK;
  }
  int64_t left = n;
  if (left >= kGraphSteps) {
    if (int rc = build_graph(c)) return rc;
    while (left >= kGraphSteps) {
      CK(cudaGraphLaunch(c->graph, c->stream), "graph launch");
      left -= kGraphSteps;
      c->last_launches += 4 * kGraphSteps;
    }
  }
  for (int64_t k = 0; k < left; ++k) {
    launch_push(c->refs, c->push_grid, c->stream);
    launch_collide(c->refs, c->collide_grid, c->stream);
    launch_finish(c->refs, 0, c->stream);
    launch_move(c->refs, c->move_grid, c->stream);
    c->last_launches += 4;
  }
  CK(cudaGetLastError(), "step");
  return SLPIC_OK;
}

int slpic_step_small(slpic_ctx* c, int64_t n, int64_t* done) {
  if (!c || n < 0 || !done) return fail(c, SLPIC_ERR_INVALID_ARG, "bad arguments");
  *done = 0;
  if (int rc = prepare(c)) return rc;
  return run_small(c, n, done);
}

int slpic_set_small_limit(slpic_ctx* c, int max_tiles) {
  if (!c || max_tiles < 0 || max_tiles > kSmallMaxTiles)
    return fail(c, SLPIC_ERR_INVALID_ARG, "small-path limit must be 0..%d tiles", kSmallMaxTiles);
  c->small_limit = max_tiles;
  return SLPIC_OK;
}

int slpic_synchronize(slpic_ctx* c) {
  if (!c) return SLPIC_ERR_INVALID_ARG;
  return sync(c);
}

int slpic_clear_error(slpic_ctx* c) {
  if (!c) return SLPIC_ERR_INVALID_ARG;
  if (!c->committed) return SLPIC_OK;
  if (int rc = set_device(c)) return rc;
  CK(cudaStreamSynchronize(c->stream), "clear");
  CK(cudaMemset(&c->d_ctrl->error, 0, sizeof(int)), "clear");
  for (int i = 0; i < c->n_inst; ++i) {
    const InstDev& P = c->h_inst[i];
    CK(cudaMemset(P.acc, 0, ACC_COUNT * 8), "clear");
    for (int s = 0; s < 2; ++s) CK(cudaMemset(P.rho_acc[s], 0, (P.n_cells + 1) * 8), "clear");
  }
  if (int rc = replan(c)) return rc;
  CK(cudaStreamSynchronize(c->stream), "clear");
  return SLPIC_OK;
}

int slpic_count(slpic_ctx* c, int inst, int species, int64_t* n) {
  if (!valid_inst(c, inst) || (species != 0 && species != 1) || !n)
    return fail(c, SLPIC_ERR_INVALID_ARG, "bad arguments");
  if (int rc = prepare(c)) return rc;
  int rc = sync(c);
  SpeciesState st;
  if (int r2 = read_state(c, inst, species, &st)) return r2;
  *n = st.n_live;
  return rc;
}

namespace {

int read_common(slpic_ctx* c, int inst, int species, const Arrays& host, int64_t capacity,
                int64_t* n_out) {
  if (!valid_inst(c, inst) || (species != 0 && species != 1) || !n_out || capacity < 0)
    return fail(c, SLPIC_ERR_INVALID_ARG, "bad arguments");
  if (int rc = precision_check(c, host.fp64)) return rc;
  if (int rc = prepare(c)) return rc;
  int rc = sync(c);
  SpeciesState st;
  if (int r2 = read_state(c, inst, species, &st)) return r2;
  *n_out = st.n_live;
  if ((int64_t)st.n_live > capacity)
    return fail(c, SLPIC_ERR_INVALID_ARG, "host buffers hold %lld markers, %u live",
                (long long)capacity, st.n_live);
  if (st.n_live > 0) {
    if (int r3 = arrays_check(c, host)) return r3;
    const SpeciesDev& S = c->h_inst[inst].sp[species];
    const SoA& d = S.buf[st.cur];
    std::vector<uint32_t> fill(st.n_tiles);
    CK(cudaMemcpy(fill.data(), S.fill[st.cur], st.n_tiles * 4, cudaMemcpyDeviceToHost), "read");
    const size_t slots = (size_t)st.n_tiles * kTile;
    std::vector<char> tmp(field_bytes(c, 1, slots));
    const void* srcs[7] = {d.cell, d.off, d.vx, d.vy, d.vz, d.wj, d.id};
    for (int f = 0; f < 7; ++f) {
      const size_t esz = field_bytes(c, f, 1);
      CK(cudaMemcpy(tmp.data(), srcs[f], slots * esz, cudaMemcpyDeviceToHost), "read");
      char* out = static_cast<char*>(host.f[f]);
      size_t o = 0;
      for (uint32_t k = 0; k < st.n_tiles; ++k) {
        std::memcpy(out + o * esz, tmp.data() + (size_t)k * kTile * esz, (size_t)fill[k] * esz);
        o += fill[k];
      }
    }
  }
  return rc;
}

}  // namespace

int slpic_read_particles(slpic_ctx* c, int inst, int species, const slpic_soa_f32* host,
                         int64_t capacity, int64_t* n_out) {
  return read_common(c, inst, species, arrays_of(host), capacity, n_out);
}

int slpic_read_particles_f64(slpic_ctx* c, int inst, int species, const slpic_soa_f64* host,
                             int64_t capacity, int64_t* n_out) {
  return read_common(c, inst, species, arrays_of(host), capacity, n_out);
}

int slpic_read_charge(slpic_ctx* c, int inst, int species, int64_t* host, int64_t n) {
  if (!valid_inst(c, inst) || (species != 0 && species != 1) || !host)
    return fail(c, SLPIC_ERR_INVALID_ARG, "bad arguments");
  if (int rc = prepare(c)) return rc;
  int rc = sync(c);
  const InstDev& P = c->h_inst[inst];
  if (n != P.n_cells + 1) return fail(c, SLPIC_ERR_INVALID_ARG, "need n_cells + 1 values");
  if (int r2 = materialize_deposit(c, inst)) return r2;
  CK(cudaMemcpy(host, P.rho_last[species], n * 8, cudaMemcpyDeviceToHost), "read charge");
  return rc;
}

int slpic_read_density(slpic_ctx* c, int inst, int species, double* host, int64_t n) {
  if (!valid_inst(c, inst) || (species != 0 && species != 1) || !host)
    return fail(c, SLPIC_ERR_INVALID_ARG, "bad arguments");
  if (int rc = prepare(c)) return rc;
  const InstDev& P = c->h_inst[inst];
  if (n != P.n_cells + 1) return fail(c, SLPIC_ERR_INVALID_ARG, "need n_cells + 1 values");
  std::vector<int64_t> q(n);
  int rc = slpic_read_charge(c, inst, species, q.data(), n);
  if (rc && rc != SLPIC_ERR_CAPACITY && rc != SLPIC_ERR_TIMEOUT) return rc;
  const double unit = std::ldexp(1.0, -P.charge_shift);
  for (int64_t k = 0; k < n; ++k) {
    const double vol = P.area * P.dx * ((k == 0 || k == n - 1) ? 0.5 : 1.0);
    host[k] = (double)q[k] * unit / vol;
  }
  return rc;
}

int slpic_read_field(slpic_ctx* c, int inst, double* phi, double* E, int64_t n) {
  if (!valid_inst(c, inst) || !phi || !E) return fail(c, SLPIC_ERR_INVALID_ARG, "bad arguments");
  if (int rc = prepare(c)) return rc;
  int rc = sync(c);
  const InstDev& P = c->h_inst[inst];
  if (n != P.n_cells + 1) return fail(c, SLPIC_ERR_INVALID_ARG, "need n_cells + 1 values");
  // the step keeps only the node field; phi is formed from the last deposit
  // (in the frozen-field mode it stays the vacuum solution)
  if (P.field_mode == 1 && c->stepped[inst]) {
    launch_phi(c->refs, inst, c->stream);
    CK(cudaGetLastError(), "read field");
    CK(cudaStreamSynchronize(c->stream), "read field");
  }
  CK(cudaMemcpy(phi, P.phi, n * 8, cudaMemcpyDeviceToHost), "read field");
  CK(cudaMemcpy(E, P.E64, n * 8, cudaMemcpyDeviceToHost), "read field");
  return rc;
}

int slpic_read_tallies(slpic_ctx* c, int inst, slpic_tallies* out) {
  static_assert(sizeof(slpic_tallies) == sizeof(TallyRec), "tally layout");
  if (!valid_inst(c, inst) || !out) return fail(c, SLPIC_ERR_INVALID_ARG, "bad arguments");
  if (int rc = prepare(c)) return rc;
  int rc = sync(c);
  CK(cudaMemcpy(out, c->h_inst[inst].total, sizeof *out, cudaMemcpyDeviceToHost), "read tallies");
  return rc;
}

int slpic_read_history(slpic_ctx* c, int inst, slpic_tallies* out, int64_t capacity,
                       int64_t* n_out) {
  if (!valid_inst(c, inst) || !out || !n_out || capacity < 0)
    return fail(c, SLPIC_ERR_INVALID_ARG, "bad arguments");
  if (int rc = prepare(c)) return rc;
  int rc = sync(c);
  InstState is;
  CK(cudaMemcpy(&is, c->d_istate + inst, sizeof is, cudaMemcpyDeviceToHost), "history");
  const InstDev& P = c->h_inst[inst];
  const long long have = std::min<long long>(is.n_steps_done, P.ring_len);
  const long long m = std::min<long long>(have, capacity);
  std::vector<TallyRec> ring(P.ring_len);
  CK(cudaMemcpy(ring.data(), P.ring, sizeof(TallyRec) * P.ring_len, cudaMemcpyDeviceToHost),
     "history");
  for (long long k = 0; k < m; ++k) {
    const long long s = is.n_steps_done - m + k;
    std::memcpy(out + k, &ring[s % P.ring_len], sizeof(TallyRec));
  }
  *n_out = m;
  return rc;
}

int slpic_read_current(slpic_ctx* c, int inst, double* Ia, double* Ic) {
  if (!valid_inst(c, inst) || !Ia || !Ic) return fail(c, SLPIC_ERR_INVALID_ARG, "bad arguments");
  slpic_tallies t;
  int64_t n = 0;
  int rc = slpic_read_history(c, inst, &t, 1, &n);
  if (n == 0) {
    *Ia = *Ic = 0;
    return rc;
  }
  const double dt = c->h_inst[inst].dt;
  // electrons leaving through the anode and ions leaving through the cathode
  // both carry conventional current in the +x direction through the gap
  *Ia = kQe * (t.w_abs[kElectron][1] - t.w_abs[kIon][1]) / dt;
  *Ic = kQe * (t.w_abs[kIon][0] - t.w_abs[kElectron][0] + t.w_see) / dt;
  return rc;
}

int slpic_read_gain(slpic_ctx* c, int inst, double* G) {
  if (!valid_inst(c, inst) || !G) return fail(c, SLPIC_ERR_INVALID_ARG, "bad arguments");
  slpic_tallies t;
  int rc = slpic_read_tallies(c, inst, &t);
  InstState is;
  CK(cudaMemcpy(&is, c->d_istate + inst, sizeof is, cudaMemcpyDeviceToHost), "gain");
  const InstDev& P = c->h_inst[inst];
  const double seed = (double)is.w_seed / P.c64.wscale;
  *G = seed > 0 ? t.w_gain_gen0 / seed : 0.0;
  return rc;
}

int slpic_set_profiling(slpic_ctx* c, int on) {
  if (!c) return SLPIC_ERR_INVALID_ARG;
  c->profiling = on != 0;
  c->ev_used = 0;
  c->prof_ms = 0;
  c->prof_launches = 0;
  return SLPIC_OK;
}

int slpic_read_profile(slpic_ctx* c, double* ms, int64_t* launches) {
  if (!c || !ms || !launches) return SLPIC_ERR_INVALID_ARG;
  if (int rc = prepare(c)) return rc;
  int rc = sync(c);
  for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
    float t = 0;
    CK(cudaEventElapsedTime(&t, c->ev[k], c->ev[k + 1]), "profile");
    c->prof_ms += t;
    c->prof_launches += 1;
  }
  c->ev_used = 0;
  *ms = c->prof_ms;
  *launches = c->prof_launches;
  return rc;
}

int slpic_read_wait_stats(slpic_ctx* c, int64_t* waits, int64_t* longest) {
  if (!c || !waits || !longest) return SLPIC_ERR_INVALID_ARG;
  if (int rc = prepare(c)) return rc;
  int rc = sync(c);
  Control h;
  CK(cudaMemcpy(&h, c->d_ctrl, sizeof h, cudaMemcpyDeviceToHost), "wait stats");
  *waits = h.spin_waits;
  *longest = h.spin_max;
  unsigned int z[2] = {0u, 0u};
  CK(cudaMemcpy(&c->d_ctrl->spin_waits, z, sizeof z, cudaMemcpyHostToDevice), "wait stats");
  return rc;
}

int slpic_launch_count(slpic_ctx* c, int64_t* launches) {
  if (!c || !launches) return SLPIC_ERR_INVALID_ARG;
  *launches = c->last_launches;
  return SLPIC_OK;
}

int slpic_philox2x32(int device, uint32_t key, const uint32_t* ctr, int64_t n,
                     uint32_t* out) {
  if (!ctr || !out || n < 0) return SLPIC_ERR_INVALID_ARG;
  if (n == 0) return SLPIC_OK;
  if (cudaSetDevice(device) != cudaSuccess) return SLPIC_ERR_CUDA;
  uint32_t *dc = nullptr, *dout = nullptr;
  const size_t b = (size_t)n * 8;
  if (cudaMalloc(&dc, b) != cudaSuccess) return SLPIC_ERR_CUDA;
  if (cudaMalloc(&dout, b) != cudaSuccess) {
    cudaFree(dc);
    return SLPIC_ERR_CUDA;
  }
  int rc = SLPIC_OK;
  if (cudaMemcpy(dc, ctr, b, cudaMemcpyHostToDevice) != cudaSuccess) rc = SLPIC_ERR_CUDA;
  if (!rc) {
    launch_philox2(key, dc, dout, n, 0);
    if (cudaGetLastError() != cudaSuccess) rc = SLPIC_ERR_CUDA;
  }
  if (!rc && cudaMemcpy(out, dout, b, cudaMemcpyDeviceToHost) != cudaSuccess) rc = SLPIC_ERR_CUDA;
  cudaFree(dc);
  cudaFree(dout);
  return rc;
}

int slpic_philox(int device, uint64_t seed, const uint32_t* ctr, int64_t n, uint32_t* out) {
  if (!ctr || !out || n < 0) return SLPIC_ERR_INVALID_ARG;
  if (n == 0) return SLPIC_OK;
  if (cudaSetDevice(device) != cudaSuccess) return SLPIC_ERR_CUDA;
  uint32_t *dc = nullptr, *dout = nullptr;
  const size_t b = (size_t)n * 16;
  if (cudaMalloc(&dc, b) != cudaSuccess) return SLPIC_ERR_CUDA;
  if (cudaMalloc(&dout, b) != cudaSuccess) {
    cudaFree(dc);
    return SLPIC_ERR_CUDA;
  }
  int rc = SLPIC_OK;
  if (cudaMemcpy(dc, ctr, b, cudaMemcpyHostToDevice) != cudaSuccess) rc = SLPIC_ERR_CUDA;
  if (!rc) {
    launch_philox((uint32_t)seed, (uint32_t)(seed >> 32), dc, dout, n, 0);
    if (cudaGetLastError() != cudaSuccess) rc = SLPIC_ERR_CUDA;
  }
  if (!rc && cudaMemcpy(out, dout, b, cudaMemcpyDeviceToHost) != cudaSuccess) rc = SLPIC_ERR_CUDA;
  cudaFree(dc);
  cudaFree(dout);
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Launch shape and its autotuner.
// ---------------------------------------------------------------------------
extern "C" int slpic_set_launch_shape(slpic_ctx* c, int push_warps, int collide_ctas_per_sm) {
  if (!c) return SLPIC_ERR_INVALID_ARG;
  if (int rc = prepare(c)) return rc;
  return apply_shape(c, push_warps, collide_ctas_per_sm);
}

extern "C" int slpic_get_launch_shape(slpic_ctx* c, int* push_warps, int* collide_ctas_per_sm) {
  if (!c || !push_warps || !collide_ctas_per_sm)
    return fail(c, SLPIC_ERR_INVALID_ARG, "NULL argument");
  if (int rc = prepare(c)) return rc;
  *push_warps = c->refs.push_warps;
  *collide_ctas_per_sm = c->collide_per_sm;
  return SLPIC_OK;
}

namespace {

// Device time per marker-step of `steps` steps of the current shape, on the
// context's own markers (the graph is built before the clock starts).
int time_shape(slpic_ctx* c, int64_t steps, double* ns_per_marker_step) {
  if (steps >= kGraphSteps)
    if (int rc = build_graph(c)) return rc;
  auto marker_steps = [&](long long* out) -> int {
    long long sum = 0;
    for (int i = 0; i < c->n_inst; ++i) {
      slpic_tallies t;
      if (int rc = slpic_read_tallies(c, i, &t)) return rc;
      sum += t.marker_steps;
    }
    *out = sum;
    return SLPIC_OK;
  };
  long long m0 = 0, m1 = 0;
  if (int rc = marker_steps(&m0)) return rc;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a), "event");
  CK(cudaEventCreate(&b), "event");
  cudaEventRecord(a, c->stream);
  int rc = slpic_step(c, steps);
  cudaEventRecord(b, c->stream);
  if (!rc) rc = sync(c);
  float ms = 0.0f;
  if (!rc && cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
    rc = fail(c, SLPIC_ERR_CUDA, "autotune: event timing");
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (!rc) rc = marker_steps(&m1);
  if (rc) return rc;
  *ns_per_marker_step = m1 > m0 ? 1e6 * ms / (double)(m1 - m0) : 1e30;
  return SLPIC_OK;
}

}  // namespace

extern "C" int slpic_autotune(slpic_ctx* c, int64_t steps_each, int* push_warps,
                              int* collide_ctas_per_sm) {
  if (!c) return SLPIC_ERR_INVALID_ARG;
  if (steps_each < 1) return fail(c, SLPIC_ERR_INVALID_ARG, "autotune: steps_each < 1");
  if (int rc = prepare(c)) return rc;
  // coordinate search: particle-kernel warps with the current collision
  // shape, then collision CTAs per SM with the best warps
  int best_w = c->refs.push_warps, best_cc = c->collide_per_sm;
  double best = 1e300;
  for (int w = 4; w <= c->max_push_warps; w += 4) {
    if (int rc = apply_shape(c, w, best_cc)) return rc;
    double t = 0;
    if (int rc = time_shape(c, steps_each, &t)) return rc;
    if (t < best) {
      best = t;
      best_w = w;
    }
  }
  const int cc_try[4] = {2, 4, 8, 16};
  for (int k = 0; k < 4; ++k) {
    if (int rc = apply_shape(c, best_w, cc_try[k])) return rc;
    double t = 0;
    if (int rc = time_shape(c, steps_each, &t)) return rc;
    if (t < best) {
      best = t;
      best_cc = cc_try[k];
    }
  }
  if (int rc = apply_shape(c, best_w, best_cc)) return rc;
  if (push_warps) *push_warps = best_w;
  if (collide_ctas_per_sm) *collide_ctas_per_sm = best_cc;
  return SLPIC_OK;
}

// ---------------------------------------------------------------------------
// Breakdown-voltage search (the batched Paschen sweep).  Host orchestration of
// the public calls: per round, set every instance's voltage, speed limit and
// step, replace its markers by the seed electrons, step the whole batch in
// chunks until every avalanche has left the gap, and shrink the brackets.
// ---------------------------------------------------------------------------
extern "C" int slpic_paschen_bisect(slpic_ctx* c, const slpic_paschen_spec* ps, double* Vb_lo,
                                    double* Vb_hi, double* gain) {
  if (!c) return SLPIC_ERR_INVALID_ARG;
  if (!ps || !Vb_lo || !Vb_hi || !ps->V_lo || !ps->V_hi)
    return fail(c, SLPIC_ERR_INVALID_ARG, "paschen: NULL argument");
  const int np = ps->n_pd, nv = ps->n_v;
  if (np < 1 || nv < 1 || (long long)np * nv != c->n_inst)
    return fail(c, SLPIC_ERR_INVALID_ARG, "paschen: the context must hold n_pd * n_v = %d instances",
                c->n_inst);
  if (ps->rounds < 1 || ps->n_seed < 1 || ps->chunk_steps < 1 || ps->max_steps < 1 ||
      !(ps->e0 >= 0))
    return fail(c, SLPIC_ERR_INVALID_ARG, "paschen: bad rounds, n_seed, e0 or step counts");
  for (int p = 0; p < np; ++p)
    if (!(ps->V_lo[p] > 0) || !(ps->V_hi[p] > ps->V_lo[p]))
      return fail(c, SLPIC_ERR_INVALID_ARG, "paschen: bracket %d is not 0 < lo < hi", p);
  // An avalanche with more than T_e = (1 + 1/gamma) n_seed live electrons, or
  // T_i = n_seed / gamma live ions, has G >= 1 for certain (every ionization
  // leaves an ion that reaches the cathode).  Electrons at most double per
  // step, so the next chunk is as long as the stores allow (at least one
  // step: 2 T_e electrons and T_i + T_e ions).
  const int n = c->n_inst;
  std::vector<int64_t> thr_e(n), thr_i(n);
  for (int i = 0; i < n; ++i) {
    if (int rc = check_config(c, i)) return rc;
    // the least yield of the instance's model
    const double g = c->hi[i].emission_model == SLPIC_EMISSION_ENERGY
                         ? 0.09 * std::pow(0.1 / 700.0, 0.05)
                         : c->hi[i].gamma;
    if (!(g > 0)) return fail(c, SLPIC_ERR_INVALID_ARG, "paschen: instance %d has gamma <= 0", i);
    thr_e[i] = (int64_t)std::ceil((1.0 + 1.0 / g) * (double)ps->n_seed);
    thr_i[i] = (int64_t)std::ceil((double)ps->n_seed / g);
    if (c->hi[i].sp[kElectron].cap < 2 * thr_e[i] ||
        c->hi[i].sp[kIon].cap < thr_i[i] + thr_e[i])
      return fail(c, SLPIC_ERR_INVALID_ARG,
                  "paschen: instance %d needs capacities of at least %lld electrons and %lld "
                  "ions (2 (1 + 1/gamma) n_seed and n_seed/gamma + (1 + 1/gamma) n_seed)",
                  i, (long long)(2 * thr_e[i]), (long long)(thr_i[i] + thr_e[i]));
  }
  if (int rc = prepare(c)) return rc;
  std::vector<double> lo(ps->V_lo, ps->V_lo + np), hi(ps->V_hi, ps->V_hi + np);
  std::vector<double> G(n, 0.0), V(n);
  std::vector<uint64_t> seed0(n);
  for (int i = 0; i < n; ++i) {
    seed0[i] = c->hi[i].seed;
  }
  std::vector<SpeciesState> st(2 * (size_t)n);
  std::vector<char> saturated(n);
  int rc = SLPIC_OK;
  for (int round = 0; round < ps->rounds && !rc; ++round) {
    // ---- configure and seed every instance --------------------------------
    for (int p = 0; p < np && !rc; ++p) {
      for (int j = 0; j < nv && !rc; ++j) {
        const int i = p * nv + j;
        const HostInst& h = c->hi[i];
        V[i] = lo[p] + (hi[p] - lo[p]) * (j + 1) / (nv + 1);
        const double dx = h.d / h.n_cells;
        double vlim = 0.0, dt;
        if (ps->vlim_factor > 0) {
          vlim = ps->vlim_factor * std::sqrt(2.0 * kQe * V[i] / h.sp[kIon].mass);
          dt = dx / vlim;
        } else {
          dt = dx / std::sqrt(2.0 * kQe * V[i] / h.sp[kElectron].mass);
        }
        const HostSpecies& se = h.sp[kElectron];
        if ((rc = slpic_set_voltage(c, i, V[i]))) break;
        if ((rc = slpic_set_species(c, i, kElectron, se.mass, se.charge, vlim, se.cap))) break;
        if ((rc = slpic_set_dt(c, i, dt))) break;
        c->hi[i].emit = 0;
        if ((rc = refresh_inst(c, i))) break;
        if ((rc = slpic_set_seed(c, i, seed0[i] + 0x9E3779B97F4A7C15ull * (uint64_t)round)))
          break;
        if ((rc = load_common(c, i, kIon, Arrays{{}, c->fp64}, 0, 0, cudaMemcpyHostToDevice))) break;
        if ((rc = load_common(c, i, kElectron, Arrays{{}, c->fp64}, 0, 0, cudaMemcpyHostToDevice))) break;
        // tallies, seeded weight and step counter start from zero every round
        if ((rc = zero_counters(c, i))) break;
        if ((rc = slpic_seed(c, i, kElectron, ps->n_seed, SLPIC_SEED_CATHODE, ps->e0, 0.0, 0.0,
                             1.0)))
          break;
        saturated[i] = 0;
      }
    }
    if (rc) break;
    // ---- step the batch until every avalanche has left the gap --------------
    int64_t k = 1;  // next chunk: no instance can outgrow its stores in it
    for (int64_t done = 0; done < ps->max_steps && !rc;) {
      // small avalanches: runs of up to chunk_steps steps in the single-CTA
      // path while no store could pass its saturation threshold inside it
      int64_t ks = 0;
      rc = run_small(c, std::min(ps->chunk_steps, ps->max_steps - done), &ks,
                     [&](int i, int64_t, int64_t) {
                       const int64_t L = (int64_t)c->small_limit * kTile;
                       return saturated[i] || (thr_e[i] >= 3 * L && thr_i[i] > 2 * L);
                     });
      if (rc) break;
      if (ks > 0) {
        k = ks;
      } else {
        k = std::min<int64_t>(k, ps->max_steps - done);
        if ((rc = slpic_step(c, k))) break;
      }
      done += k;
      if ((rc = sync(c))) break;
      if (cudaMemcpy(st.data(), c->d_sstate, sizeof(SpeciesState) * st.size(),
                     cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = fail(c, SLPIC_ERR_CUDA, "paschen: reading the live counts");
        break;
      }
      bool live = false;
      k = ps->chunk_steps;
      for (int i = 0; i < n && !rc; ++i) {
        if (saturated[i]) continue;
        const int64_t ne = st[2 * i].n_live, ni = st[2 * i + 1].n_live;
        // above breakdown for certain; stop this avalanche before it can
        // outgrow the stores
        if (ne > thr_e[i] || ni >= thr_i[i]) {
          saturated[i] = 1;
          rc = load_common(c, i, kIon, Arrays{{}, c->fp64}, 0, 0, cudaMemcpyHostToDevice);
          if (!rc)
            rc = load_common(c, i, kElectron, Arrays{{}, c->fp64}, 0, 0, cudaMemcpyHostToDevice);
          continue;
        }
        if (ne || ni) live = true;
        // in s steps the electrons grow at most to ne 2^s and the ions to
        // ni + ne (2^s - 1)
        if (ne > 0) {
          const int64_t ce = c->hi[i].sp[kElectron].cap, ci = c->hi[i].sp[kIon].cap;
          int64_t s = 1;  // grows while s + 1 steps stay inside both stores
          while (s < k && s < 30 && ne * (int64_t(2) << s) <= ce &&
                 ni + ne * ((int64_t(2) << s) - 1) <= ci)
            ++s;
          k = std::min(k, s);
        }
      }
      if (!live) break;
    }
    if (rc) break;
    // ---- gains and brackets -------------------------------------------------
    for (int i = 0; i < n && !rc; ++i) {
      if (saturated[i]) {
        G[i] = std::numeric_limits<double>::infinity();
        continue;
      }
      slpic_tallies t;
      if ((rc = slpic_read_tallies(c, i, &t))) break;
      InstState is;
      if (cudaMemcpy(&is, c->d_istate + i, sizeof is, cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = fail(c, SLPIC_ERR_CUDA, "paschen: reading the seeded weight");
        break;
      }
      const double w_seed = (double)is.w_seed / c->h_inst[i].c64.wscale;
      G[i] = w_seed > 0 ? t.w_gain_gen0 / w_seed : 0.0;
    }
    if (rc) break;
    for (int p = 0; p < np; ++p) {
      int j = 0;
      while (j < nv && !(G[p * nv + j] >= 1.0)) ++j;
      const double a = j == 0 ? lo[p] : V[p * nv + j - 1];
      const double b = j == nv ? hi[p] : V[p * nv + j];
      lo[p] = a;
      hi[p] = b;
    }
  }
  for (int i = 0; i < n; ++i) {
    c->hi[i].emit = 1;
    const int r2 = refresh_inst(c, i);
    if (!rc) rc = r2;
  }
  if (rc) return rc;
  for (int p = 0; p < np; ++p) {
    Vb_lo[p] = lo[p];
    Vb_hi[p] = hi[p];
  }
  if (gain)
    for (int i = 0; i < n; ++i) gain[i] = G[i];
  return SLPIC_OK;
}

// ---------------------------------------------------------------------------
// The paper's breakdown test (Sec. V): the trend of the ion population.
// ---------------------------------------------------------------------------
// Advance every instance by n steps: the single-CTA path while it applies,
// then the batched kernels.
int advance(slpic_ctx* c, int64_t n) {
  for (int64_t done = 0; done < n;) {
    int64_t k = 0;
    if (int rc = run_small(c, n - done, &k)) return rc;
    if (k == 0) {
      k = n - done;
      if (int rc = slpic_step(c, k)) return rc;
    }
    done += k;
  }
  return SLPIC_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint and resume.  A snapshot is a host byte buffer:
//   header  "SLPICSV1", version, precision, n_inst;
//   per instance: its record (cells, ring length, whether it has stepped,
//     the counters of InstState, the tally totals, live markers and next id
//     per species), then the history ring, phi, E (FP64), E (FP32), the last
//     deposit of both species, and the live markers of each species in store
//     order as seven arrays (cell, offset, vx, vy, vz, w_j, id), every array
//     padded to 8 bytes.
namespace {
struct SnapHeader {
  char magic[8];
  int32_t version;
  int32_t fp64;
  int32_t n_inst;
  int32_t pad;
};
struct SnapInst {
  int32_t n_cells;
  int32_t ring_len;
  int32_t stepped;
  int32_t pad;
  InstState is;
  TallyRec total;
  uint64_t n_live[2];
  uint32_t next_id[2];
};
constexpr char kSnapMagic[8] = {'S', 'L', 'P', 'I', 'C', 'S', 'V', '1'};
size_t pad8(size_t b) { return (b + 7) & ~size_t(7); }

// Bytes of instance i's part of a snapshot (the live counts are read).
int snap_inst_bytes(slpic_ctx* c, int i, const SpeciesState st[2], size_t* bytes) {
  const InstDev& P = c->h_inst[i];
  const size_t nn = (size_t)P.n_cells + 1;
  size_t b = pad8(sizeof(SnapInst)) + pad8(sizeof(TallyRec) * P.ring_len) + 2 * nn * 8 +
             pad8(nn * 4) + 2 * nn * 8;
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < 7; ++k) b += pad8(field_bytes(c, k, st[s].n_live));
  *bytes = b;
  return SLPIC_OK;
}
}  // namespace

extern "C" int slpic_save(slpic_ctx* c, void* buf, size_t capacity, size_t* size_out) {
  if (!c || !size_out) return SLPIC_ERR_INVALID_ARG;
  if (int rc = prepare(c)) return rc;
  if (int rc = sync(c)) return rc;
  const int n = c->n_inst;
  std::vector<SpeciesState> st(2 * (size_t)n);
  size_t total = pad8(sizeof(SnapHeader));
  for (int i = 0; i < n; ++i) {
    // the deposit and phi as a read would form them
    if (int rc = materialize_deposit(c, i)) return rc;
    if (c->h_inst[i].field_mode == 1 && c->stepped[i]) {
      launch_phi(c->refs, i, c->stream);
      CK(cudaGetLastError(), "save");
    }
    for (int s = 0; s < 2; ++s)
      if (int rc = read_state(c, i, s, &st[2 * i + s])) return rc;
    size_t b = 0;
    snap_inst_bytes(c, i, &st[2 * i], &b);
    total += b;
  }
  CK(cudaStreamSynchronize(c->stream), "save");
  *size_out = total;
  if (!buf) return SLPIC_OK;
  if (capacity < total)
    return fail(c, SLPIC_ERR_CAPACITY, "save: the snapshot takes %zu bytes, the buffer %zu",
                total, capacity);
  char* o = static_cast<char*>(buf);
  SnapHeader h{};
  std::memcpy(h.magic, kSnapMagic, 8);
  h.version = 1;
  h.fp64 = c->fp64;
  h.n_inst = n;
  std::memcpy(o, &h, sizeof h);
  o += pad8(sizeof h);
  for (int i = 0; i < n; ++i) {
    const InstDev& P = c->h_inst[i];
    const size_t nn = (size_t)P.n_cells + 1;
    SnapInst r{};
    r.n_cells = P.n_cells;
    r.ring_len = P.ring_len;
    r.stepped = c->stepped[i];
    CK(cudaMemcpy(&r.is, c->d_istate + i, sizeof r.is, cudaMemcpyDeviceToHost), "save");
    CK(cudaMemcpy(&r.total, P.total, sizeof r.total, cudaMemcpyDeviceToHost), "save");
    for (int s = 0; s < 2; ++s) {
      r.n_live[s] = st[2 * i + s].n_live;
      r.next_id[s] = st[2 * i + s].next_id;
    }
    std::memcpy(o, &r, sizeof r);
    o += pad8(sizeof r);
    CK(cudaMemcpy(o, P.ring, sizeof(TallyRec) * P.ring_len, cudaMemcpyDeviceToHost), "save");
    o += pad8(sizeof(TallyRec) * P.ring_len);
    CK(cudaMemcpy(o, P.phi, nn * 8, cudaMemcpyDeviceToHost), "save");
    o += nn * 8;
    CK(cudaMemcpy(o, P.E64, nn * 8, cudaMemcpyDeviceToHost), "save");
    o += nn * 8;
    CK(cudaMemcpy(o, P.E32, nn * 4, cudaMemcpyDeviceToHost), "save");
    o += pad8(nn * 4);
    for (int s = 0; s < 2; ++s) {
      CK(cudaMemcpy(o, P.rho_last[s], nn * 8, cudaMemcpyDeviceToHost), "save");
      o += nn * 8;
    }
    for (int s = 0; s < 2; ++s) {
      const int64_t nl = st[2 * i + s].n_live;
      Arrays a{};
      a.fp64 = c->fp64;
      char* base = o;
      for (int k = 0; k < 7; ++k) {
        a.f[k] = base;
        base += pad8(field_bytes(c, k, nl));
      }
      int64_t got = 0;
      if (int rc = read_common(c, i, s, a, nl, &got)) return rc;
      o = base;
    }
  }
  return SLPIC_OK;
}

extern "C" int slpic_load(slpic_ctx* c, const void* buf, size_t size) {
  if (!c || !buf) return SLPIC_ERR_INVALID_ARG;
  const char* o = static_cast<const char*>(buf);
  const char* end = o + size;
  SnapHeader h;
  if (size < sizeof h) return fail(c, SLPIC_ERR_INVALID_ARG, "load: not a snapshot");
  std::memcpy(&h, o, sizeof h);
  if (std::memcmp(h.magic, kSnapMagic, 8) != 0 || h.version != 1)
    return fail(c, SLPIC_ERR_INVALID_ARG, "load: not a snapshot of this library");
  if (h.fp64 != c->fp64 || h.n_inst != c->n_inst)
    return fail(c, SLPIC_ERR_INVALID_ARG,
                "load: snapshot of %d instances in FP%d, context of %d in FP%d", h.n_inst,
                h.fp64 ? 64 : 32, c->n_inst, c->fp64 ? 64 : 32);
  if (int rc = prepare(c)) return rc;
  if (int rc = sync(c)) return rc;
  o += pad8(sizeof h);
  for (int i = 0; i < c->n_inst; ++i) {
    const InstDev& P = c->h_inst[i];
    const size_t nn = (size_t)P.n_cells + 1;
    SnapInst r;
    if (end - o < (ptrdiff_t)sizeof r) return fail(c, SLPIC_ERR_INVALID_ARG, "load: truncated");
    std::memcpy(&r, o, sizeof r);
    if (r.n_cells != P.n_cells || r.ring_len != P.ring_len)
      return fail(c, SLPIC_ERR_INVALID_ARG,
                  "load: instance %d has %d cells in the snapshot, %d in the context", i,
                  r.n_cells, P.n_cells);
    SpeciesState st[2];
    for (int s = 0; s < 2; ++s) st[s].n_live = (uint32_t)r.n_live[s];
    size_t b = 0;
    snap_inst_bytes(c, i, st, &b);
    if ((size_t)(end - o) < b) return fail(c, SLPIC_ERR_INVALID_ARG, "load: truncated");
    o += pad8(sizeof r);
    const char* ring = o;
    o += pad8(sizeof(TallyRec) * P.ring_len);
    const char* phi = o;
    o += nn * 8;
    const char* e64 = o;
    o += nn * 8;
    const char* e32 = o;
    o += pad8(nn * 4);
    const char* rho[2];
    for (int s = 0; s < 2; ++s) {
      rho[s] = o;
      o += nn * 8;
    }
    for (int s = 0; s < 2; ++s) {
      const int64_t nl = (int64_t)r.n_live[s];
      Arrays a{};
      a.fp64 = c->fp64;
      for (int k = 0; k < 7; ++k) {
        a.f[k] = const_cast<char*>(o);
        o += pad8(field_bytes(c, k, nl));
      }
      if (int rc = load_common(c, i, s, a, nl, r.next_id[s], cudaMemcpyHostToDevice)) return rc;
    }
    // the counters, tallies, field and deposit as saved (the loads above
    // set the seeded and live weights from the markers)
    CK(cudaMemcpy(c->d_istate + i, &r.is, sizeof r.is, cudaMemcpyHostToDevice), "load");
    CK(cudaMemcpy(P.total, &r.total, sizeof r.total, cudaMemcpyHostToDevice), "load");
    CK(cudaMemcpy(P.ring, ring, sizeof(TallyRec) * P.ring_len, cudaMemcpyHostToDevice), "load");
    CK(cudaMemcpy(P.phi, phi, nn * 8, cudaMemcpyHostToDevice), "load");
    CK(cudaMemcpy(P.E64, e64, nn * 8, cudaMemcpyHostToDevice), "load");
    CK(cudaMemcpy(P.E32, e32, nn * 4, cudaMemcpyHostToDevice), "load");
    for (int s = 0; s < 2; ++s)
      CK(cudaMemcpy(P.rho_last[s], rho[s], nn * 8, cudaMemcpyHostToDevice), "load");
    c->stepped[i] = (char)r.stepped;
    c->dep_dirty[i] = 0;
  }
  if (int rc = replan(c)) return rc;
  return sync(c);
}

extern "C" int slpic_set_spin_limit(slpic_ctx* c, uint32_t polls) {
  if (!c) return SLPIC_ERR_INVALID_ARG;
  c->spin_limit = polls;
  if (!c->d_ctrl) return SLPIC_OK;
  if (int rc = set_device(c)) return rc;
  CK(cudaStreamSynchronize(c->stream), "spin limit");
  CK(cudaMemcpy(&c->d_ctrl->spin_limit, &polls, sizeof polls, cudaMemcpyHostToDevice),
     "spin limit");
  return SLPIC_OK;
}

extern "C" int slpic_test_skip_barrier(slpic_ctx* c, int inst, int64_t barrier) {
  if (!c) return SLPIC_ERR_INVALID_ARG;
  if (inst < -1 || inst >= c->n_inst || barrier < 0)
    return fail(c, SLPIC_ERR_INVALID_ARG, "skip barrier: instance in [-1, n_inst), barrier >= 0");
  if (int rc = prepare(c)) return rc;
  CK(cudaStreamSynchronize(c->stream), "skip barrier");
  const int cta = inst + 1;
  const long long b = inst < 0 ? 0 : (long long)barrier;
  CK(cudaMemcpy(&c->d_ctrl->skip_cta, &cta, sizeof cta, cudaMemcpyHostToDevice), "skip barrier");
  CK(cudaMemcpy(&c->d_ctrl->skip_barrier, &b, sizeof b, cudaMemcpyHostToDevice), "skip barrier");
  return SLPIC_OK;
}

extern "C" int slpic_multiplication(slpic_ctx* c, int64_t steps_per_window, int n_windows,
                                    double* see, double* M) {
  if (!c) return SLPIC_ERR_INVALID_ARG;
  if (!see || steps_per_window < 1 || n_windows < 1)
    return fail(c, SLPIC_ERR_INVALID_ARG, "multiplication: need see, steps_per_window >= 1 "
                                          "and n_windows >= 1");
  if (int rc = prepare(c)) return rc;
  const int n = c->n_inst;
  // flux weight emitted at the cathode so far, from the step's FP64 totals
  std::vector<double> w0(n), w1(n);
  auto read_see = [&](std::vector<double>& out) -> int {
    for (int i = 0; i < n; ++i) {
      slpic_tallies t;
      if (int rc = slpic_read_tallies(c, i, &t)) return rc;
      out[i] = t.w_see;
    }
    return SLPIC_OK;
  };
  if (int rc = read_see(w0)) return rc;
  for (int w = 0; w < n_windows; ++w) {
    if (int rc = advance(c, steps_per_window)) return rc;
    if (int rc = read_see(w1)) return rc;
    for (int i = 0; i < n; ++i) see[(size_t)i * n_windows + w] = w1[i] - w0[i];
    w0 = w1;
  }
  if (M) {
    for (int i = 0; i < n; ++i) {
      const double* S = see + (size_t)i * n_windows;
      for (int k = 1; k < n_windows; ++k)
        M[(size_t)i * (n_windows - 1) + k - 1] =
            S[k - 1] > 0.0 ? S[k] / S[k - 1] : std::numeric_limits<double>::quiet_NaN();
    }
  }
  return SLPIC_OK;
}

extern "C" int slpic_ion_trend(slpic_ctx* c, int64_t steps_per_window, int n_windows,
                               double* means, int* above) {
  if (!c) return SLPIC_ERR_INVALID_ARG;
  if (!means || steps_per_window < 1 || n_windows < 2)
    return fail(c, SLPIC_ERR_INVALID_ARG, "ion trend: need means, steps_per_window >= 1 and "
                                          "n_windows >= 2");
  if (int rc = prepare(c)) return rc;
  const int n = c->n_inst;
  std::vector<SpeciesState> st(2 * (size_t)n);
  std::vector<InstState> is(n);
  std::vector<char> stopped(n, 0);
  auto read_states = [&]() -> int {
    if (int rc = sync(c)) return rc;
    if (cudaMemcpy(st.data(), c->d_sstate, sizeof(SpeciesState) * st.size(),
                   cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(is.data(), c->d_istate, sizeof(InstState) * is.size(),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(c, SLPIC_ERR_CUDA, "ion trend: reading the live counts");
    return SLPIC_OK;
  };
  if (int rc = read_states()) return rc;
  for (int w = 0; w < n_windows; ++w) {
    // live ions summed over the window's steps, from the per-step running sum
    std::vector<long long> ion0(n);
    for (int i = 0; i < n; ++i) ion0[i] = is[i].ion_steps;
    for (int64_t done = 0; done < steps_per_window;) {
      // every instance is above breakdown for certain: nothing left to follow
      if (std::all_of(stopped.begin(), stopped.end(), [](char x) { return x != 0; })) break;
      // small populations: whole runs of steps in the single-CTA path, which
      // stops by itself before a store outgrows it
      int64_t k = 0;
      if (int rc = run_small(c, steps_per_window - done, &k)) return rc;
      if (k == 0) {
        // chunk length: per step the electrons grow at most to 2 e + i
        // (ionization and emission) and the ions to i + e, so both stay below
        // 3^k (e + i) after k steps; keep that inside the smaller store
        k = steps_per_window - done;
        for (int i = 0; i < n; ++i) {
          if (stopped[i]) continue;
          const int64_t m = (int64_t)st[2 * i].n_live + st[2 * i + 1].n_live;
          if (m == 0) continue;
          const int64_t cap = std::min(c->hi[i].sp[kElectron].cap, c->hi[i].sp[kIon].cap);
          int64_t s = 0, grow = m;
          while (s < k && grow * 3 <= cap && s < 36) {
            grow *= 3;
            ++s;
          }
          k = std::min(k, std::max<int64_t>(s, 1));
        }
        if (int rc = slpic_step(c, k)) return rc;
      }
      done += k;
      if (int rc = read_states()) return rc;
      for (int i = 0; i < n; ++i) {
        if (stopped[i]) continue;
        const int64_t e = st[2 * i].n_live, ni = st[2 * i + 1].n_live;
        // the population has grown past a third of the smaller store (the
        // next step could overflow it): above breakdown
        if (3 * (e + ni) > std::min(c->hi[i].sp[kElectron].cap, c->hi[i].sp[kIon].cap)) {
          stopped[i] = 1;
          int rc = load_common(c, i, kIon, Arrays{{}, c->fp64}, 0, 0, cudaMemcpyHostToDevice);
          if (!rc)
            rc = load_common(c, i, kElectron, Arrays{{}, c->fp64}, 0, 0, cudaMemcpyHostToDevice);
          if (rc) return rc;
          st[2 * i].n_live = st[2 * i + 1].n_live = 0;
        }
      }
    }
    for (int i = 0; i < n; ++i)
      means[(size_t)i * n_windows + w] =
          stopped[i] ? -1.0 : (double)(is[i].ion_steps - ion0[i]) / (double)steps_per_window;
  }
  if (above) {
    for (int i = 0; i < n; ++i) {
      const double* m = means + (size_t)i * n_windows;
      bool grows = stopped[i] != 0;
      if (!grows) {
        grows = m[n_windows - 1] > 0.0;
        for (int w = 0; w + 1 < n_windows; ++w) grows = grows && m[n_windows - 1] > m[w];
      }
      above[i] = grows ? 1 : 0;
    }
  }
  return SLPIC_OK;
}

// ---------------------------------------------------------------------------
// slpic_philox_static: the Philox self-check without device allocation.  The
// counters (first half) and the outputs (second half) live in one file-scope
// device array of the module.  Callers that cannot allocate: a process whose
// memory pool already holds the whole device, or one checking the random
// stream while a simulation runs on another stream (the cudaFree of
// slpic_philox would synchronise the device under it).

static __device__ __align__(256) uint32_t g_philox_scratch[2 * 4 * SLPIC_PHILOX_STATIC_MAX];

namespace {
constexpr int kStaticMaxDevices = 64;

// Per device: the array's address and a private non-blocking stream, valid in
// the context they were made in.
struct StaticScratch {
  CUcontext ctx = nullptr;
  uint32_t* ptr = nullptr;
  cudaStream_t stream = nullptr;
};
std::mutex g_scratch_mu;
StaticScratch g_scratch[kStaticMaxDevices];

// The driver's cuCtxGetCurrent, found through the runtime (no link to the
// driver library).
using CtxGetCurrent = CUresult (*)(CUcontext*);
CtxGetCurrent ctx_get_current() {
  static CtxGetCurrent fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<CtxGetCurrent>(f);
  }();
  return fn;
}
}  // namespace

// Set-up for `device`, which must be current: the array's address
// (cudaGetSymbolAddress, which loads the module's device data if CUDA has not
// yet done so), a private non-blocking stream, and the load of the Philox
// kernel's module.  Cached per device, and redone when the device's current
// context differs from the one the cache was made in (after cudaDeviceReset);
// the stream of a context that is gone is not touched again.
int philox_static_setup(int device, StaticScratch* out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  CUcontext cur = nullptr;
  CtxGetCurrent get = ctx_get_current();
  if (!get || get(&cur) != CUDA_SUCCESS || !cur)
    return fail(nullptr, SLPIC_ERR_CUDA, "slpic_philox_static: no current context on device %d",
                device);
  StaticScratch& s = g_scratch[device];
  if (!(s.ptr && s.ctx == cur)) {
    uint32_t* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&p, g_philox_scratch);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "slpic_philox_static: cudaGetSymbolAddress");
    cudaStream_t st = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "slpic_philox_static: stream");
    e = (cudaError_t)philox_preload();
    if (e != cudaSuccess) {
      cudaStreamDestroy(st);
      return cuda_fail(nullptr, e, "slpic_philox_static: kernel load");
    }
    s.ctx = cur;
    s.ptr = p;
    s.stream = st;
  }
  *out = s;
  return SLPIC_OK;
}

extern "C" int slpic_philox_static(int device, uint64_t seed, const uint32_t* ctr, int64_t n,
                                   uint32_t* out) {
  if (!ctr || !out || n < 0)
    return fail(nullptr, SLPIC_ERR_INVALID_ARG, "slpic_philox_static: NULL array or n < 0");
  if (n > SLPIC_PHILOX_STATIC_MAX)
    return fail(nullptr, SLPIC_ERR_INVALID_ARG,
                "slpic_philox_static: n = %lld counters exceeds SLPIC_PHILOX_STATIC_MAX = %d "
                "(the size of its fixed scratch); use slpic_philox or split the call",
                (long long)n, SLPIC_PHILOX_STATIC_MAX);
  if (device < 0 || device >= kStaticMaxDevices)
    return fail(nullptr, SLPIC_ERR_INVALID_ARG, "slpic_philox_static: device %d out of range",
                device);
  if (n == 0) return SLPIC_OK;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "slpic_philox_static: cudaSetDevice");
  StaticScratch sc;
  if (int rc = philox_static_setup(device, &sc)) return rc;
  uint32_t* dctr = sc.ptr;
  uint32_t* dout = sc.ptr + 4 * (size_t)SLPIC_PHILOX_STATIC_MAX;
  const size_t b = (size_t)n * 16;
  e = cudaMemcpyAsync(dctr, ctr, b, cudaMemcpyHostToDevice, sc.stream);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "slpic_philox_static: counters to device");
  launch_philox((uint32_t)seed, (uint32_t)(seed >> 32), dctr, dout, n, sc.stream);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "slpic_philox_static: launch");
  e = cudaMemcpyAsync(out, dout, b, cudaMemcpyDeviceToHost, sc.stream);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "slpic_philox_static: outputs to host");
  e = cudaStreamSynchronize(sc.stream);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "slpic_philox_static: synchronise");
  return SLPIC_OK;
}


// slpic_philox_static's set-up for `device` from slpic_create; the calling
// thread's current device is restored.
int philox_static_setup_for(int device) {
  if (device < 0 || device >= kStaticMaxDevices) return SLPIC_OK;
  int prev = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "slpic_create: cudaGetDevice");
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "slpic_create: cudaSetDevice");
  StaticScratch sc;
  int rc = philox_static_setup(device, &sc);
  cudaSetDevice(prev);
  return rc;
}
