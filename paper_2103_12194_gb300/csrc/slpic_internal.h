// Internal device-side layout shared by the kernels and the host driver of
// libslpic.  Nothing here is part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace slpic {

constexpr int kElectron = 0;
constexpr int kIon = 1;
constexpr uint32_t kGenBit = 0x80000000u;
constexpr uint32_t kSerialMask = 0x7FFFFFFFu;
constexpr uint32_t kSeedStep = 0xFFFFFFFFu;

// Marker stores are sequences of tiles of kTile slots.  The particle kernel
// gives every tile to one warp (kPerLane slots per lane: lane l holds slots
// l, l + 32, ...); a CTA of up to kPushMaxWarps warps takes super-tiles of
// one tile per warp, and each warp streams its tiles through kPushStages
// shared-memory stages.
constexpr int kTile = 128;
constexpr int kPerLane = kTile / 32;
constexpr int kPushMaxWarps = 20;
constexpr int kPushStages = 2;
// The particle kernel advances a lane's kPerLane slots in kHalves passes.
constexpr int kHalves = 2;
constexpr int kPerHalf = kPerLane / kHalves;
// Shared-memory stage of one tile: cell and id (4 bytes each), then the five
// real streams (off, vx, vy, vz, w_j) of sizeof(R) bytes.
template <typename R>
__host__ __device__ constexpr int stage_bytes() {
  return kTile * (8 + 5 * (int)sizeof(R));
}
// Relative cost of a super-tile of each species in the particle kernel's
// static split of the super-tiles over the CTAs (ions draw no collision test).
constexpr unsigned int kWeightElectron = 3;
constexpr unsigned int kWeightIon = 2;

// Device error word values (copied to the host status codes).
constexpr int kErrNone = 0;
constexpr int kErrCapacity = 1;
constexpr int kErrTimeout = 2;
constexpr int kErrIdWrap = 3;

// Bounded waits: polls before a wait gives up with kErrTimeout (each poll of
// an mbarrier suspends the thread for up to about a microsecond), unless the
// context sets another limit (Control::spin_limit).
constexpr uint32_t kSpinLimit = 1u << 22;

// Per-step accumulators of one instance (integer; weights in fixed point).
enum Acc : int {
  ACC_CAND = 0,
  ACC_COLL0,  // elastic
  ACC_COLL1,  // excitation
  ACC_COLL2,  // ionization
  ACC_SEE,
  ACC_NABS,        // 4 entries: [species][electrode]
  ACC_WABS = ACC_NABS + 4,
  ACC_WSEE = ACC_WABS + 4,
  ACC_WIONZ,
  ACC_WCATH,
  ACC_WCATH0,
  ACC_CLAMP,
  ACC_MAJ,
  ACC_MSTEPS,
  ACC_GWCATH0,  // yield * w_j of first-generation ions at the cathode
  ACC_COUNT
};

// Record of one step, converted (same layout as slpic_tallies).
struct TallyRec {
  long long step;
  long long n_live[2];
  double w_live[2];
  long long n_coll[3];
  long long n_candidates;
  long long n_abs[2][2];
  double w_abs[2][2];
  long long n_see;
  double w_see;
  double w_ionz;
  double w_cath_ion;
  double w_cath_ion_gen0;
  long long n_clamp;
  long long n_majorant;
  long long marker_steps;
  double w_gain_gen0;
};

// Structure-of-arrays marker store in the arithmetic type R of the marker
// path (float in FP32 contexts, double in FP64 contexts).  The device
// descriptors hold the float view; kernels of an FP64 context take the double
// view of the same pointers.
template <typename R>
struct SoAT {
  int32_t* cell;
  R* off;
  R* vx;
  R* vy;
  R* vz;
  R* wj;
  uint32_t* id;
};
using SoA = SoAT<float>;

template <typename R>
__host__ __device__ inline SoAT<R> soa_as(const SoA& s) {
  return SoAT<R>{s.cell, reinterpret_cast<R*>(s.off), reinterpret_cast<R*>(s.vx),
                 reinterpret_cast<R*>(s.vy), reinterpret_cast<R*>(s.vz),
                 reinterpret_cast<R*>(s.wj), s.id};
}

// Processes of an electron collision: elastic, up to three excitation
// levels, ionization.
constexpr int kMaxExc = 3;
constexpr int kMaxProc = kMaxExc + 2;

// One node of the FP64 cross-section table: the cumulative cross sections of
// the processes in order, and a pad.
struct alignas(64) TabNode64 {
  double s[kMaxProc];
  double pad[8 - kMaxProc];
};

// Constants of the step in the marker path's arithmetic type R; the host
// derives both sets from the same double-precision configuration.
template <typename R>
struct StepConsts {
  R qmdt[2];      // (q / m) dt per species
  R vlim[2];      // speed limit per species (+inf: beta = 1)
  R K_V[2];       // 2 e / m: speed^2 per eV, per species
  R dtdx;         // dt / dx
  R K_E;          // m_e / (2 e): eV per (m/s)^2
  R ndt;          // n_g dt
  R P0;           // null-collision majorant probability
  R vb_cap;       // cap of beta v in the majorant
  R R2;           // 2 m_e / M
  R e_ex[kMaxExc];  // excitation thresholds [eV]
  R e_io;           // ionization threshold [eV]
  R sigT_ion;     // sqrt(k T / M)
  R K_Ei;         // M / (2 e): eV per (m/s)^2 of an ion
  R gamma;        // secondary-emission yield
  R wscale;       // 2^charge_shift
  R two_pi;
  R e_lo, e_hi;   // table range [eV]
};

// Marker store of one (instance, species): a sequence of tiles of kTile
// slots; tile k holds fill[k] live markers in its first slots, in order.  The
// particle kernel compacts each tile in place (no dependence between tiles);
// births are appended after the last live marker; when the tiles become
// sparse the whole store is repacked into the other buffer.
//
// Mutable per-(instance, species) state, resident on the device.
struct SpeciesState {
  uint32_t cur;       // buffer holding the markers
  uint32_t n_tiles;   // tiles in use
  uint32_t n_live;    // live markers (sum of the fills)
  uint32_t next_id;   // next serial number
};

// Repacking of one segment at the end of a step (decided by k_finish,
// done by k_move).
struct Transfer {
  uint32_t compact;       // repack the tiles of buffer src into buffer dst
  uint32_t src, dst;
  uint32_t n_tiles_old;   // tiles to repack
  uint32_t n_new;         // live markers after the step
  uint32_t tail;          // first slot the step's births went to
  uint32_t end;           // one past the last birth
  uint32_t pad;
};

// A null-collision candidate as the particle kernel leaves it: the electron's
// state after its push and its slot in the tile after compaction (the top bit
// marks an ionization once it has collided; vx then holds the energy given to
// the secondary).  One record fills a 32-byte sector in float, so the
// collision kernel reads a candidate with one sector instead of one per field.
template <typename R>
struct CandRec;
template <>
struct alignas(32) CandRec<float> {
  int cell;
  float off, vx, vy, vz, wj;
  uint32_t id, slot;
};
template <>
struct alignas(16) CandRec<double> {
  int cell;
  uint32_t id;
  double off, vx, vy, vz, wj;
  uint32_t slot, pad;
};
static_assert(sizeof(CandRec<float>) == 32, "one sector per float record");
constexpr uint32_t kIonizedMark = 0x80000000u;

// Configuration of one species of one instance (constant during a run).
struct SpeciesDev {
  SoA buf[2];         // tiled marker store (cap_tiles * kTile slots each)
  uint32_t* fill[2];  // [cap_tiles] live markers per tile of each buffer
  SoA stage_b;        // electrons only: emission births, slot = ion tile * kTile + rank
  uint32_t* births;   // ions: [cap_tiles] electrons emitted by each tile in the step
  void* crec;         // electrons: [cap_tiles * kTile] CandRec<R>, the tile's
                      // null-collision candidates in slot order
  uint32_t* n_cand;   // electrons: [cap_tiles] candidates per tile
  uint32_t cap_tiles;
  uint32_t pad;
};

// Configuration of one instance (constant during a run).
struct InstDev {
  int n_cells;
  int field_mode;
  int charge_shift;
  int tab_lo_exp2;
  int tab_log2_sub;
  int tab_nodes;      // real nodes (a padding node follows)
  uint32_t key0, key1;
  uint32_t ctr_inst;  // counter word 2 = ctr_inst * 2 + species
  uint32_t key2;      // Philox2x32 key of the null-collision draw
  int n_exc;          // excitation levels (1..kMaxExc)
  int tab_stride;     // float4s per node of the FP32 table (1, or 2 with more levels)
  int emission_model; // 0: constant gamma; 1: Eq. sey
  int emit;           // 0: tally the yield, emit no electron
  StepConsts<float> c32;
  StepConsts<double> c64;
  double dx, d, V, area, dt;
  double pois_C;      // e dx 2^-shift / (area eps0)
  const float4* table;          // FP32: cumulative cross sections per node, n_exc + 2 of them, in tab_stride float4s
  const TabNode64* table64;     // FP64: the same in double
  float* E32;                   // node field used by the FP32 push
  double* phi;                  // node potential
  double* E64;                  // node field
  long long* pois_I;            // [nn] I_k = sum_{0<j<k} net_j of the last solve
  double* pois_D1;              // [1] D_1 of the last solve
  unsigned long long* rho_acc[2];  // fixed-point deposit of the current step
  long long* rho_last[2];          // deposit of the last finished step
  unsigned long long* acc;         // ACC_COUNT per-step accumulators
  TallyRec* ring;                  // per-step records
  TallyRec* total;                 // sums since the last reset
  int ring_len;
  int pad;
  SpeciesDev sp[2];
};

// Mutable per-instance counters.
struct InstState {
  uint32_t step;        // step index (Philox counter word 1)
  uint32_t pad;
  long long n_steps_done;
  unsigned long long w_seed;     // fixed-point sum of seeded electron weights
  unsigned long long w_live[2];  // fixed-point sum of live weights per species
  long long ion_steps;           // sum over the steps of the live ions after each
};

// Global state of the batched step.
struct Control {
  unsigned int epoch;        // step epoch of the look-back records
  unsigned int n_super;      // particle-kernel super-tiles this step
  unsigned int w_total;      // their summed weights
  unsigned int n_seg;        // segments = instances * 2
  unsigned int finish_done;  // CTAs of the finish kernel that completed
  int error;                 // first device error (kErr*)
  int error_inst;
  unsigned int spin_waits;   // polls that found data not yet there
  unsigned int spin_max;     // longest single wait, in polls
  unsigned int coll_counter; // next collision chunk to hand out
  unsigned int n_coll_chunks;
  unsigned int move_counter; // next repacking chunk to hand out
  unsigned int n_move_chunks;
  unsigned int small_bar;    // single-CTA path: arrivals at its grid barriers
  int small_stop;            // single-CTA path: a store outgrew it
  long long small_done;      // single-CTA path: steps run by the last launch
  unsigned int spin_limit;   // polls before a bounded wait gives up (0: kSpinLimit)
  int skip_cta;              // test hook: CTA + 1 of the single-CTA path that skips
  long long skip_barrier;    //   its arrival at this grid barrier (0: none)
};

// Look-back record of one chunk of an ordered scan.
struct ChunkStatus {
  unsigned int flag;  // (epoch << 2) | state; state 1 = aggregate, 2 = inclusive
  unsigned int agg;
  unsigned int incl;
  unsigned int pad;
};

// Collision chunks: kCollWarps warps of T / kCollWarps consecutive tiles
// each.  Electron chunks have T = coll_tiles[inst] tiles, a power of two in
// [kCollMinChunkTiles, kCollMaxChunkTiles] chosen from the instance's last
// step so that a warp meets about kCollTargetPerWarp candidates (many
// collisions per step: small chunks, more warps); ion chunks (the electrons
// emitted at the cathode, rare) have kCollMaxChunkTiles.  Repacking chunks:
// kMoveChunkTiles tiles.
constexpr int kCollWarps = 8;
constexpr int kCollMaxChunkTiles = kCollWarps * 32;
constexpr int kCollMinChunkTiles = kCollWarps;
constexpr int kCollTargetPerWarp = 256;
constexpr int kMoveChunkTiles = 128;
// Single-CTA path (small.cu): at most this many tiles per store and instance
// when a step starts.
constexpr int kSmallMaxTiles = 32;

struct DeviceRefs {
  InstDev* inst;          // [n_inst]
  InstState* istate;      // [n_inst]
  SpeciesState* sstate;   // [n_inst * 2]
  Transfer* xfer;         // [n_inst * 2]
  Control* ctrl;
  unsigned int* seg_start;   // [n_seg + 1] first super-tile of each segment
  unsigned int* seg_wstart;  // [n_seg + 1] summed super-tile weights before each segment
  unsigned int* coll_start;  // [n_inst + 1] first collision chunk of each instance
  unsigned int* coll_tiles;  // [n_inst] tiles per electron collision chunk
  unsigned int* move_start;  // [n_seg + 1] first repacking chunk of each segment
  ChunkStatus* coll_scan;    // [max collision chunks]
  ChunkStatus* move_scan;    // [max repacking chunks]
  int n_inst;
  int smem_nodes;         // deposit grid nodes in shared memory (0: global atomics)
  int push_warps;         // warps per particle-kernel CTA = tiles per super-tile
  int fp64;               // marker path in double precision (else float)
  int finish_net_nodes;   // k_finish keeps the net deposit of up to this many nodes in shared memory
};

// Launchers (defined in the .cu files).
void launch_push(const DeviceRefs& r, int grid, cudaStream_t s);
// Particle-kernel shape for a shared-memory deposit grid of smem_nodes nodes:
// warps per CTA, resident CTAs per SM and dynamic shared memory per CTA.
int push_config(int fp64, int smem_nodes, int* warps, int* blocks_per_sm, size_t* smem_bytes);
// Resident particle-kernel CTAs per SM for `warps` warps per CTA.
int push_blocks_per_sm(int fp64, int warps, int smem_nodes, int* blocks_per_sm);
// mode 0: finish a step and plan the next; mode 1: plan only (one CTA).
void launch_finish(const DeviceRefs& r, int mode, cudaStream_t s);
// Shared-memory room of k_finish for the largest grid (0: read from global).
int finish_config(int max_nodes, int* net_nodes);
void launch_move(const DeviceRefs& r, int grid, cudaStream_t s);
// Node potential of instance inst from its last deposit (Poisson mode).
void launch_phi(const DeviceRefs& r, int inst, cudaStream_t s);
// Deposit of instance inst's live markers (n_tiles tiles of both species)
// added to its last-step grids; used with an imposed field, where the step
// itself deposits nothing.
void launch_deposit(const DeviceRefs& r, int inst, int n_tiles, cudaStream_t s);
// Scatter the null-collision candidates queued by the particle kernel.
void launch_collide(const DeviceRefs& r, int grid, cudaStream_t s);
int collide_config();
// Seeding: n markers written contiguously from slot `base` of the current
// buffer; mode 0/1/2 as SLPIC_SEED_*; for mode 3 (thermal) e0 carries the
// thermal speed sqrt(k T / m).
void launch_seed(const DeviceRefs& r, int inst, int species, uint32_t base, uint32_t first_id,
                 uint32_t n, int mode, double e0, double e_lo, double lr, double wj,
                 cudaStream_t s);
void launch_validate(int fp64, const SoA& d, uint32_t n, int N, int shift, unsigned int* bad,
                     unsigned long long* wsum, cudaStream_t s);
int philox_preload();
void launch_philox(uint32_t k0, uint32_t k1, const uint32_t* ctr, uint32_t* out,
                   long long n, cudaStream_t s);
void launch_philox2(uint32_t k, const uint32_t* ctr, uint32_t* out, long long n,
                    cudaStream_t s);
// Single-CTA path: shared memory for field-mode-1 grids of up to
// max_poisson_nodes nodes and resident CTAs per SM (0: does not fit); then up
// to n_steps steps of every instance (one CTA each), stopping before a step
// when a store has more than max_tiles tiles.  Steps run: Control::small_done.
int small_config(int fp64, int max_poisson_nodes, size_t* smem_bytes, int* blocks_per_sm);
int launch_small(const DeviceRefs& r, long long n_steps, int max_tiles, size_t smem_bytes,
                 cudaStream_t s);

}  // namespace slpic
