// SLPIC-MCC oracle: a plain, slow CPU restatement of one speed-limited
// particle-in-cell step with Monte-Carlo collisions (Theis, Werner, Jenkins,
// Cary, "Computing the Paschen curve for argon with speed-limited
// particle-in-cell simulation").
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
// call this file: only the tests, the package's smoke check and the CPU
// baseline leg of the benchmark use it.  It shares no code, header, constant
// or table generator with the CUDA library.
//
// Everything is written as loops over markers in array order, one marker at a
// time, in the order the method states.  The arithmetic type R is double for
// the reference (FP64) mode and float for the FP32 mirror mode; the mirror
// evaluates the same expressions left to right in IEEE single precision
// (build with -ffp-contract=off so that no multiply-add is fused), which is
// what lets counts and deposits be compared bit for bit against an FP32
// implementation that makes the same choices.
//
// Readings of the paper that this file fixes (the paper is silent on them):
//  * cathode at x = 0 with phi = 0, anode at x = d with phi = V (Sec. IV);
//  * linear (cloud-in-cell) shape for gather and deposit (Eq. Ansatz);
//  * the kick solves Eq. slpicEOMv exactly over the step with E_x held at
//    its gathered value (leapfrog below the speed limit; across and above it
//    the motion is unlimited in the time tau = integral of beta dt, and the
//    step's end follows from the elapsed time, a closed form in asinh); the
//    drift uses beta of the post-kick speed (Eqs. slpicEOMx, slpicEOMv,
//    betaAbrupt).  The FP64 reference evaluates that solution directly; the
//    FP32 mirror restates the library's single-precision solution of the same
//    equation;
//  * collision probability of a marker per step = beta v dt / lambda_mfp
//    = n_g sigma(eps) beta v dt (Sec. III, the d'/lambda_mfp rule and
//    Eq. SLPICcollisionNumber with beta_n = 1, whole-marker collisions),
//    realised with a null-collision majorant: a candidate draw u < P0 every
//    step (Philox2x32-10), then the process from a second draw;
//  * Vahedi-Surendra elastic angles, isotropic excitation with the threshold
//    removed, ionization with a uniform split of the excess energy (the
//    Kutasi sharing rule is not given in the paper), Ar+ born with a gas
//    temperature Maxwellian;
//  * secondary-emission yield either constant (gamma, the Lieberman value of
//    Sec. V) or the energy-dependent yield of Eq. sey (Sec. IV) evaluated at
//    the ion's kinetic energy when it crosses the cathode; the expected yield
//    of first-generation ions is tallied for the gain.
//
// Parity unpinned: the ensemble quantities (Townsend alpha of the synthetic
// gas, multiplication, breakdown voltage) have no printed value in the paper;
// they are pinned only by closed forms and self-consistency checks.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <type_traits>
#include <vector>

namespace {

// CODATA 2018 constants (SI).
const double kQe = 1.602176634e-19;     // elementary charge [C]
const double kMe = 9.1093837015e-31;    // electron mass [kg]
const double kKB = 1.380649e-23;        // Boltzmann constant [J/K]
const double kEps0 = 8.8541878128e-12;  // vacuum permittivity [F/m]
const double kTwoPi = 6.283185307179586;

const int ELECTRON = 0;
const int ION = 1;
const uint32_t GEN_BIT = 0x80000000u;   // set on markers of later generations
const uint32_t SEED_STEP = 0xFFFFFFFFu; // Philox "step" word used for seeding

// ---------------------------------------------------------------------------
// Philox4x32-10, from its published definition (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two
// 32x32->64 multiplies with the round keys bumped by the Weyl constants.
// ---------------------------------------------------------------------------
void philox4x32_10(const uint32_t ctr_in[4], uint32_t k0, uint32_t k1,
                   uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Philox2x32-10 from the same publication: ten rounds of one 32x32->64
// multiply, the round key bumped by the Weyl constant.
void philox2x32_10(const uint32_t ctr_in[2], uint32_t k, uint32_t out[2]) {
  const uint32_t M = 0xD256D193u, W = 0x9E3779B9u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) k += W;
    uint64_t p = (uint64_t)M * (uint64_t)c0;
    uint32_t hi = (uint32_t)(p >> 32), lo = (uint32_t)p;
    uint32_t n0 = hi ^ c1 ^ k;
    uint32_t n1 = lo;
    c0 = n0; c1 = n1;
  }
  out[0] = c0; out[1] = c1;
}

// 32 random bits -> uniform in (0, 1): (floor(x / 2^9) + 1/2) / 2^23.  The
// result has at most 24 significant bits, so it is the same number in float
// and in double.
template <typename R>
R uniform01(uint32_t x) {
  return ((R)(x >> 9) + (R)0.5) * (R)(1.0 / 8388608.0);
}

template <typename R>
struct Marker {
  int32_t cell;
  R off;  // position inside the cell, in [0, 1)
  R vx, vy, vz;
  R wj;   // flux weight w_j = w_p / beta (constant along a trajectory)
  uint32_t id;
};

}  // namespace

extern "C" {

// Configuration of one instance (one gap at one (p, V)).  Mirrors nothing in
// the CUDA library; the tests fill it from the same numbers they give the
// library.
typedef struct {
  int n_cells;
  double d;          // gap [m]
  double V;          // anode potential [V]
  double area;       // electrode area that the 1D weights refer to [m^2]
  int field_mode;    // 0: vacuum field -V/d kept fixed, 1: Poisson every step
  double p_Pa, T_K;  // background argon
  double dt;         // time step [s]
  double mass[2];    // [kg] electron, ion
  double charge[2];  // [C]
  double vlim[2];    // speed limit [m/s]; <= 0 or inf means beta = 1
  double gamma_se;   // ion-induced secondary-electron yield at the cathode
  int charge_shift;  // fixed-point scale: charge unit = 2^-shift flux weight
  uint64_t seed;
  uint32_t instance;
  int tab_lo_exp2;   // table starts at 2^tab_lo_exp2 eV
  int tab_log2_sub;  // 2^tab_log2_sub nodes per octave
  int tab_octaves;   // table spans this many octaves
  const float* sig_el;  // cross sections at the nodes [m^2]
  const float* sig_ex;
  const float* sig_io;
  double e_ex, e_io;    // excitation and ionization thresholds [eV]
  int precision;        // 64: FP64 reference, 32: FP32 mirror
  int emission_model;   // 0: constant gamma_se; 1: Eq. sey
  int emit;             // 0: tally the yield but emit no electron
  int n_exc;            // excitation levels (1..3): sig_ex/e_ex, then these
  const float* sig_ex2;
  const float* sig_ex3;
  double e_ex2, e_ex3;
  int kick_scheme;      // 0: Eq. slpicEOMv solved exactly; 1: a planted
                        // trapezoid-rule approximation (pins only)
} oracle_config;

// Per-step record of what happened (all sums over markers, in the step).
typedef struct {
  int64_t step;
  int64_t n_live[2];       // live markers after the step
  double w_live[2];        // sum of w_j of live markers after the step
  int64_t n_coll[3];       // elastic, excitation, ionization
  int64_t n_candidates;    // null-collision candidates (u1 < P0)
  int64_t n_abs[2][2];     // [species][0: cathode, 1: anode]
  double w_abs[2][2];
  int64_t n_see;           // secondary electrons emitted
  double w_see;
  double w_ionz;           // sum of w_j of ionizing electrons
  double w_cath_ion;       // sum of w_j of ions absorbed at the cathode
  double w_cath_ion_gen0;  // same, ions of the first generation only
  int64_t n_clamp;         // energies clamped at 0 after an inelastic event
  int64_t n_majorant;      // markers whose beta*v exceeded the table's cap
  int64_t marker_steps;    // markers pushed in the step
  double w_gain_gen0;      // sum of yield * w_j over first-generation ions at the cathode
} oracle_tally;

}  // extern "C"

namespace {

template <typename R>
struct Sim {
  oracle_config cfg;
  int N = 0;
  int n_nodes_tab = 0;
  std::vector<Marker<R>> sp[2];
  uint32_t next_id[2] = {0, 0};
  uint32_t step = 0;
  // tables: cumulative cross sections of the processes in order (elastic,
  // the excitation levels, ionization), in R
  int n_exc = 1, n_proc = 3;
  std::vector<R> S[5];
  // field at the nodes (FP64 solution, and its R copy used by the push)
  std::vector<double> phi, E64;
  std::vector<R> E;
  std::vector<int64_t> charge[2];  // deposit of the last step (fixed point)
  std::vector<oracle_tally> history;
  // derived constants, in R
  R qmdt[2], dtdx, vlim[2], K_E, K_V[2], ndt, P0, vb_cap, R2, e_ex[3], e_io;
  R sigT_ion, gamma, two_pi, wscale, K_Ei;
  bool limited[2];

  void init(const oracle_config& c) {
    cfg = c;
    N = c.n_cells;
    const double dx = c.d / c.n_cells;
    for (int s = 0; s < 2; ++s) {
      qmdt[s] = (R)((c.charge[s] / c.mass[s]) * c.dt);
      limited[s] = c.vlim[s] > 0.0 && std::isfinite(c.vlim[s]);
      vlim[s] = limited[s] ? (R)c.vlim[s] : std::numeric_limits<R>::infinity();
      K_V[s] = (R)(2.0 * kQe / c.mass[s]);
    }
    dtdx = (R)(c.dt / dx);
    K_E = (R)(0.5 * c.mass[ELECTRON] / kQe);
    const double n_g = c.p_Pa / (kKB * c.T_K);
    ndt = (R)(n_g * c.dt);
    R2 = (R)(2.0 * c.mass[ELECTRON] / c.mass[ION]);
    n_exc = c.n_exc >= 1 && c.n_exc <= 3 ? c.n_exc : 1;
    n_proc = n_exc + 2;
    e_ex[0] = (R)c.e_ex;
    e_ex[1] = (R)c.e_ex2;
    e_ex[2] = (R)c.e_ex3;
    e_io = (R)c.e_io;
    sigT_ion = (R)std::sqrt(kKB * c.T_K / c.mass[ION]);
    gamma = (R)c.gamma_se;
    K_Ei = (R)(0.5 * c.mass[ION] / kQe);  // eV per (m/s)^2 of an ion
    two_pi = (R)kTwoPi;
    wscale = (R)std::ldexp(1.0, c.charge_shift);

    // Cumulative cross sections at the nodes, plus one padding node equal to
    // the last so that interpolation at the top node reads a valid neighbour.
    n_nodes_tab = (c.tab_octaves << c.tab_log2_sub) + 1;
    const float* part[5] = {c.sig_el, c.sig_ex, c.sig_ex2, c.sig_ex3, nullptr};
    part[n_exc + 1] = c.sig_io;
    for (int k = 0; k < n_proc; ++k) S[k].assign(n_nodes_tab + 1, 0);
    R smax = 0;
    for (int j = 0; j < n_nodes_tab; ++j) {
      S[0][j] = (R)part[0][j];
      for (int k = 1; k < n_proc; ++k) S[k][j] = S[k - 1][j] + (R)part[k][j];
      smax = std::max(smax, S[n_proc - 1][j]);
    }
    for (int k = 0; k < n_proc; ++k) S[k][n_nodes_tab] = S[k][n_nodes_tab - 1];
    // Majorant of n_g sigma_tot(eps) min(v, vlim) dt over the table.  Above
    // the table's top energy the cross sections are held at the top node and
    // beta*v is capped at the speed of that energy (only matters for beta=1).
    R e_top = (R)std::ldexp(1.0, c.tab_lo_exp2 + c.tab_octaves);
    R v_top = std::sqrt(e_top * K_V[ELECTRON]);
    vb_cap = std::min(vlim[ELECTRON], v_top);
    P0 = (ndt * vb_cap) * smax;

    phi.assign(N + 1, 0.0);
    E64.assign(N + 1, -c.V / c.d);
    for (int k = 0; k <= N; ++k) phi[k] = c.V * k / N;
    E.assign(N + 1, (R)(-c.V / c.d));
    charge[0].assign(N + 1, 0);
    charge[1].assign(N + 1, 0);
  }

  // The null-collision draw of an electron in a step: word 0 of
  // Philox2x32-10 with counter (id, step) and a key mixing both seed words
  // and the instance.
  R collision_draw(uint32_t id, uint32_t stp) const {
    uint32_t ctr[2] = {id, stp}, out[2];
    const uint32_t key = (uint32_t)cfg.seed ^ (uint32_t)(cfg.seed >> 32) ^
                         (0x85EBCA6Bu * (cfg.instance + 1u));
    philox2x32_10(ctr, key, out);
    return uniform01<R>(out[0]);
  }

  void draws(uint32_t id, uint32_t stp, int species, uint32_t block,
             R u[4]) const {
    uint32_t ctr[4] = {id, stp, cfg.instance * 2u + (uint32_t)species, block};
    uint32_t out[4];
    philox4x32_10(ctr, (uint32_t)cfg.seed, (uint32_t)(cfg.seed >> 32), out);
    for (int i = 0; i < 4; ++i) u[i] = uniform01<R>(out[i]);
  }

  // Secondary-electron yield of an ion crossing the cathode: constant, or
  // Eq. sey at the ion's kinetic energy eps_i [eV] (exponent 0.05 below
  // 700 eV, 0.72 from 700 eV on).
  R yield(const Marker<R>& m) const {
    if (cfg.emission_model != 1) return gamma;
    const R eps_i = (m.vx * m.vx + m.vy * m.vy + m.vz * m.vz) * K_Ei;
    const R expo = eps_i < (R)700 ? (R)0.05 : (R)0.72;
    return (R)0.09 * std::pow(eps_i / (R)700, expo);
  }

  // beta(v) = min(1, vlim / v), Eq. betaAbrupt.
  R beta(R v, int s) const { return v > vlim[s] ? vlim[s] / v : (R)1; }

  // New v_x after the kick of one step, A = q E_x dt / m the unlimited
  // velocity increment (Eq. slpicEOMv: dv_x/dt = beta(|v|) q E_x / m, with
  // v_y and v_z unchanged and E_x held at its gathered value over the step).
  // FP64 reference: the exact solution (kick_reference); FP32 mirror: the
  // arithmetic of the library's kick, operation by operation (kick_mirror);
  // kick_scheme 1 plants a trapezoid-rule approximation for the pins.
  R kick(const Marker<R>& m, R A, int s) const {
    if (!limited[s]) return m.vx + A;
    if (cfg.kick_scheme == 1) return kick_trapezoid(m.vx, m.vy, m.vz, A, vlim[s]);
    if constexpr (std::is_same<R, double>::value) {
      return kick_reference(m.vx, m.vy, m.vz, A, vlim[s]);
    } else {
      return kick_mirror(m.vx, m.vy, m.vz, A, vlim[s]);
    }
  }

  // Psi(w) = integral from 0 to w of max(L, sqrt(w'^2 + p^2)) dw', an odd
  // function of w.  With sqrt(w^2 + p^2) >= L for |w| >= q = sqrt(L^2 - p^2)
  // (q = 0 when p >= L):
  //   |w| <= q:  L w;
  //   |w| >  q:  sign(w) [L q + (Phi(|w|) - Phi(q)) / 2],
  // Phi(x) = x sqrt(x^2 + p^2) + p^2 asinh(x / p), the antiderivative of
  // 2 sqrt(x^2 + p^2) (Phi(x) = x^2 when p = 0).
  static double psi(double w, double p, double L) {
    const double a = std::fabs(w);
    const double sg = w < 0.0 ? -1.0 : 1.0;
    auto Phi = [p](double x) {
      if (p == 0.0) return x * x;
      return x * std::sqrt(x * x + p * p) + p * p * std::asinh(x / p);
    };
    const double q = p < L ? std::sqrt(L * L - p * p) : 0.0;
    if (a <= q) return sg * L * a;
    return sg * (L * q + 0.5 * (Phi(a) - Phi(q)));
  }

  // The exact kick (FP64 reference).  In the time tau = integral of beta dt
  // the motion of Eq. slpicEOMv is unlimited: v_x = v_x0 + a tau, a = A / dt.
  // The elapsed time is dt = integral of dtau / beta(|v|)
  // = integral of max(1, |v| / L) dtau.  With w = v_x sign(A) the speed along
  // the force and dtau = dw / |a|, the step's end w1 solves
  //   Psi(w1) - Psi(w0) = L |a| dt = L |A|.
  // Psi is increasing (slope max(L, |v|) >= L), and the root lies in
  // [w0, w0 + |A|] (tau <= dt).  It is found by Newton steps kept inside
  // that bracket (a bisection whenever a step would leave it), until the
  // bracket or the step is at the last bits of w.  Below the limit at both
  // ends of the step the motion is unlimited and the kick is v_x + A.
  static double kick_reference(double vx, double vy, double vz, double A, double L) {
    const double p2 = vy * vy + vz * vz;
    const double vt = vx + A;
    if (std::sqrt(vx * vx + p2) <= L && std::sqrt(vt * vt + p2) <= L) return vt;
    if (A == 0.0) return vx;
    const double g = A > 0.0 ? 1.0 : -1.0;
    const double p = std::sqrt(p2);
    const double w0 = g * vx;
    const double target = psi(w0, p, L) + L * std::fabs(A);
    double lo = w0, hi = w0 + std::fabs(A);
    double w = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
      const double G = psi(w, p, L) - target;
      if (G == 0.0) return g * w;
      if (G < 0.0) lo = w;
      else hi = w;
      const double slope = std::max(L, std::sqrt(w * w + p2));
      double wn = w - G / slope;
      if (!(wn > lo && wn < hi)) wn = 0.5 * (lo + hi);
      const double tol = 4.0 * std::numeric_limits<double>::epsilon() *
                         std::max(std::fabs(w), std::max(L, p));
      if (hi - lo <= tol || std::fabs(wn - w) <= 0.25 * tol) {
        w = wn;
        break;
      }
      w = wn;
    }
    return g * w;
  }

  // A planted mistake for the pins (kick_scheme 1): the elapsed time of the
  // speed-limited part taken by the trapezoid rule from the two end speeds,
  // solved by one Newton step, and a path that dips below the limit inside
  // the step treated as limited throughout.  Its errors reach tens of per
  // cent off the field axis.
  static R kick_trapezoid(R vx, R vy, R vz, R A, R L) {
    const R sp = std::sqrt(vx * vx + vy * vy + vz * vz);
    if (sp <= L) {
      const R vt = vx + A;
      if (std::sqrt(vt * vt + vy * vy + vz * vz) <= L) return vt;
    }
    const R g = A > (R)0 ? (R)1 : (R)-1;
    const R aA = g * A;
    const R p2 = vy * vy + vz * vz;
    R f, s1, v1;
    if (sp < L) {
      const R q = std::sqrt(std::max((R)0, L * L - p2));
      f = std::min((R)1, std::max((R)0, (R)1 - (q - g * vx) / aA));
      s1 = L;
      v1 = q;
    } else {
      f = (R)1;
      s1 = sp;
      v1 = g * vx;
    }
    const R K = (R)2 * f * aA * L;
    const R c = s1 + v1;
    R z = (std::sqrt(c * c + (R)4 * K) - c) * (R)0.5;
    if (z * s1 > K) z = K / s1;
    const R w = v1 + z;
    const R sn = std::sqrt(w * w + p2);
    const R t = s1 + sn;
    const R den = t * sn + z * w;
    if (den > (R)0) z = std::max((R)0, z - (z * t - K) * sn / den);
    return g * (v1 + z);
  }

  // ---- FP32 mirror of the library's kick --------------------------------
  // The library solves the same equation as kick_reference with IEEE single
  // operations only (+ - * / sqrt and fused multiply-adds), so that this
  // restatement reproduces it bit for bit.  Along the force the path has up
  // to three parts: limited and slowing (w < -q), unlimited (|w| <= q, the
  // time-integral is L dw), limited and speeding up (w > q).  In a limited
  // part, with m = |w| and D(m0, m) = integral of sqrt(x^2 + p^2) dx from
  // m0 to m = [m s - m0 s0 + p^2 log((m + s) / (m0 + s0))] / 2, the end
  // solves D(m0, m) = T (T = +-the remaining budget): a third-order series
  // guess in X = T / s0^2 (beyond |X| = 1/2, sqrt(m0^2 + 2T)), then Halley
  // steps kept inside a bracket until the step is below 2^-8 of the speed
  // (the error left is then about the cube of that, under a float ulp).
  static float mad32(float a, float b, float c) { return std::fmaf(a, b, c); }

  // Natural logarithm of a positive normal float by Tang's table-driven
  // method (ACM TOMS 16, 1990), from IEEE operations and a table:
  // y = 2^k m with m's bit pattern in [0x3F350000, 0x3FB50000) (about
  // [0.707, 1.414)); interval j of m (the top 6 bits of its offset from the
  // lower end) has centre c_j = the float at 0x3F350000 + 2^17 j + 2^16;
  // r_j = 1 / c_j rounded to float, n_j = -log(r_j) rounded to float;
  // f = m r_j - 1 in one rounding (|f| < 2^-7); log(1 + f) by its Taylor
  // series to f^4; log y = k log 2 + n_j + log(1 + f), with log 2 split in
  // two parts so that k log 2 keeps its precision.
  struct LogTable {
    float r[64], n[64];
    LogTable() {
      for (int j = 0; j < 64; ++j) {
        const uint32_t cb = 0x3F350000u + ((uint32_t)j << 17) + (1u << 16);
        float c;
        std::memcpy(&c, &cb, 4);
        r[j] = 1.0f / c;
        n[j] = (float)(-std::log((double)r[j]));
      }
    }
  };
  static float log_mirror(float y) {
    static const LogTable tab;
    uint32_t b;
    std::memcpy(&b, &y, 4);
    const int32_t ix = (int32_t)b - (int32_t)0x3F350000;
    const int32_t k = ix >> 23;
    const uint32_t mb = (uint32_t)ix & 0x7FFFFFu;
    const uint32_t bits = mb + 0x3F350000u;
    float m;
    std::memcpy(&m, &bits, 4);
    const int j = (int)(mb >> 17);
    const float f = mad32(m, tab.r[j], -1.0f);
    float q = mad32(f, -0.25f, 1.0f / 3.0f);
    q = mad32(f, q, -0.5f);
    const float lp = mad32(f * f, q, f);
    const float kf = (float)k;
    return mad32(kf, 0.693145751953125f, mad32(kf, 1.428606765330187e-06f, tab.n[j] + lp));
  }

  // End speed m >= 0 along the force with D(m0, m) = T, root in [lo, hi];
  // speeding up (fwd), the upper end is m0 + T / s0 (s >= s0 along the way),
  // with 1 / s0 from the reciprocal shared with 1 / (m0 + s0).
  static float kick_solve_mirror(float m0, float T, float lo, float hi, float p2, bool fwd) {
    const float s0 = std::sqrt(mad32(m0, m0, p2));
    const float h0 = m0 + s0;
    const float rr = 1.0f / (s0 * h0);
    const float is0 = h0 * rr, ih0 = s0 * rr;
    if (fwd) hi = mad32(T, is0, m0);
    const float X = (T * is0) * is0;
    const float c0 = m0 * is0;
    float m;
    if (std::fabs(X) <= 0.5f) {
      const float c3 = mad32(4.0f * c0, c0, -1.0f) * (float)(1.0 / 6.0);
      const float zh = X * mad32(X, mad32(X, c3, -0.5f * c0), 1.0f);
      m = mad32(s0, zh, m0);
    } else {
      m = std::sqrt(std::max(0.0f, mad32(m0, m0, T + T)));
    }
    m = std::min(std::max(m, lo), hi);
    const float hm0s0 = 0.5f * (m0 * s0);
    const float hp2 = 0.5f * p2;
    for (int it = 0; it < 24; ++it) {
      const float s = std::sqrt(mad32(m, m, p2));
      const float lg = p2 > 0.0f ? log_mirror((m + s) * ih0) : 0.0f;
      const float F = mad32(hp2, lg, mad32(0.5f * m, s, -hm0s0)) - T;
      if (F > 0.0f) hi = m;
      else lo = m;
      const float s2 = s * s;
      const float dm = ((F + F) * s2) / mad32(s2 + s2, s, -(F * m));
      float mn = m - dm;
      if (!(mn >= lo && mn <= hi)) mn = 0.5f * (lo + hi);
      const float step = m - mn;
      m = mn;
      if (std::fabs(step) <= 0.00390625f * s) break;
    }
    return m;
  }

  static float kick_mirror(float vx, float vy, float vz, float A, float L) {
    const float L2 = L * L;
    const float p2 = mad32(vy, vy, vz * vz);
    const float vt = vx + A;
    if (mad32(vx, vx, p2) <= L2 && mad32(vt, vt, p2) <= L2) return vt;
    if (!(A != 0.0f)) return vx;
    const float g = A > 0.0f ? 1.0f : -1.0f;
    float W = L * (g * A);
    float w = g * vx;
    const float q2 = L2 - p2;
    const float q = q2 > 0.0f ? std::sqrt(q2) : 0.0f;
    float m0, T, lo, hi, sgn;
    if (w < -q) {
      // limited, slowing down: the cost of reaching the unlimited zone
      // (or the axis) is D(q, |w|) >= L (|w| - q)
      m0 = -w;
      bool stay = W <= L * (m0 - q);
      if (!stay) {
        const float s0 = std::sqrt(mad32(m0, m0, p2));
        const float sq = q > 0.0f ? L : std::sqrt(p2);
        float C1 = 0.5f * (m0 * s0 - q * sq);
        if (p2 > 0.0f) C1 = mad32(0.5f * p2, log_mirror((m0 + s0) / (q + sq)), C1);
        stay = W < C1;
        if (!stay) {
          W = W - C1;
          w = -q;
        }
      }
      if (stay) {
        T = -W;
        lo = q;
        hi = m0;
        sgn = -1.0f;
        return g * (sgn * kick_solve_mirror(m0, T, lo, hi, p2, false));
      }
    }
    if (w < q) {
      // unlimited zone
      const float reach = L * (q - w);
      if (W <= reach) return g * (w + W / L);
      W = W - reach;
      w = q;
    }
    // limited, speeding up
    m0 = w;
    T = W;
    lo = w;
    hi = 0.0f;  // set by the solve
    sgn = 1.0f;
    return g * (sgn * kick_solve_mirror(m0, T, lo, hi, p2, true));
  }

  // Linear interpolation of the cumulative cross sections at eps.  Nodes sit
  // at 2^(lo + o) (1 + m / 2^sub) eV: 2^sub equal steps inside each octave.
  void xsec(R eps, R* s) const {
    const int L = cfg.tab_lo_exp2, sub = cfg.tab_log2_sub;
    const R e_lo = (R)std::ldexp(1.0, L);
    const R e_hi = (R)std::ldexp(1.0, L + cfg.tab_octaves);
    int j;
    R t;
    if (!(eps >= e_lo)) {
      j = 0;
      t = 0;
    } else if (eps >= e_hi) {
      j = n_nodes_tab - 1;
      t = 0;
    } else {
      int ex;
      R m = std::frexp(eps, &ex);  // eps = m 2^ex, m in [1/2, 1)
      int octave = ex - 1 - L;
      R pos = (m + m - (R)1) * (R)(1 << sub);  // in [0, 2^sub), exact
      R fl = std::floor(pos);
      j = (octave << sub) + (int)fl;
      t = pos - fl;
    }
    for (int k = 0; k < n_proc; ++k) s[k] = S[k][j] + t * (S[k][j + 1] - S[k][j]);
  }

  // Isotropic direction with cos(theta) = 1 - 2 ua about x, phi = 2 pi ub.
  void isotropic(R speed, R ua, R ub, R& vx, R& vy, R& vz) const {
    R ct = (R)1 - (R)2 * ua;
    R st = std::sqrt(std::max((R)0, ((R)1 - ct) * ((R)1 + ct)));
    R ph = two_pi * ub;
    vx = speed * ct;
    vy = speed * (st * std::cos(ph));
    vz = speed * (st * std::sin(ph));
  }

  // Rotate the unit vector (ux, uy, uz) by polar angle chi (given by its
  // cosine and sine) and azimuth phi about itself.  The perpendicular basis is
  // built from the x axis, or from the z axis when |ux| > 0.99.
  void rotate(R& ux, R& uy, R& uz, R cc, R sc, R cp, R sp) const {
    R nx, ny, nz;
    if (std::fabs(ux) <= (R)0.99) {
      R w = std::sqrt(((R)1 - ux) * ((R)1 + ux));
      nx = ux * cc + sc * (cp * w);
      ny = uy * cc + sc * ((uz * sp - ux * (uy * cp)) / w);
      nz = uz * cc - sc * ((uy * sp + ux * (uz * cp)) / w);
    } else {
      R w = std::sqrt(((R)1 - uz) * ((R)1 + uz));
      nx = ux * cc + sc * ((uy * sp - uz * (ux * cp)) / w);
      ny = uy * cc - sc * ((ux * sp + uz * (uy * cp)) / w);
      nz = uz * cc + sc * (cp * w);
    }
    ux = nx; uy = ny; uz = nz;
  }

  void deposit_one(const Marker<R>& m, int s, std::vector<int64_t>& q) const {
    R v = std::sqrt(m.vx * m.vx + m.vy * m.vy + m.vz * m.vz);
    R wp = beta(v, s) * m.wj;  // density weight w_p = beta w_j
    int64_t Q = (int64_t)std::llrint(wp * wscale);
    int64_t f = (int64_t)(m.off * (R)16777216.0);  // 24-bit CIC fraction
    int64_t right = (Q * f) >> 24;
    q[m.cell] += Q - right;
    q[m.cell + 1] += right;
  }

  void solve_field() {
    // (phi[k+1] - 2 phi[k] + phi[k-1]) / dx^2 = -rho_k / eps0, k = 1..N-1,
    // phi[0] = 0, phi[N] = V; Thomas algorithm on the tridiagonal system.
    const double dx = cfg.d / N;
    const double unit = std::ldexp(1.0, -cfg.charge_shift);
    std::vector<double> rhs(N + 1, 0.0), cp(N + 1, 0.0), dp(N + 1, 0.0);
    for (int k = 1; k < N; ++k) {
      double net = (double)(charge[ION][k] - charge[ELECTRON][k]);
      double rho = kQe * net * unit / (cfg.area * dx);
      rhs[k] = -rho * dx * dx / kEps0;
    }
    rhs[1] -= 0.0;       // phi[0]
    rhs[N - 1] -= cfg.V; // phi[N]
    // forward sweep: a = 1, b = -2, c = 1
    cp[1] = 1.0 / -2.0;
    dp[1] = rhs[1] / -2.0;
    for (int k = 2; k < N; ++k) {
      double den = -2.0 - cp[k - 1];
      cp[k] = 1.0 / den;
      dp[k] = (rhs[k] - dp[k - 1]) / den;
    }
    phi[0] = 0.0;
    phi[N] = cfg.V;
    if (N >= 2) {
      phi[N - 1] = dp[N - 1];
      for (int k = N - 2; k >= 1; --k) phi[k] = dp[k] - cp[k] * phi[k + 1];
    }
    E64[0] = -(phi[1] - phi[0]) / dx;
    E64[N] = -(phi[N] - phi[N - 1]) / dx;
    for (int k = 1; k < N; ++k) E64[k] = -(phi[k + 1] - phi[k - 1]) / (2.0 * dx);
    for (int k = 0; k <= N; ++k) E[k] = (R)E64[k];
  }

  void one_step() {
    oracle_tally t;
    std::memset(&t, 0, sizeof(t));
    t.step = step;
    const uint32_t s_now = step;
    std::vector<Marker<R>> born_e_ionz, born_i, born_e_see;
    for (int s = 0; s < 2; ++s) {
      std::vector<Marker<R>> survivors;
      survivors.reserve(sp[s].size());
      for (size_t i = 0; i < sp[s].size(); ++i) {
        Marker<R> m = sp[s][i];
        t.marker_steps++;
        // Field at the marker (linear interpolation between its nodes).
        R Ex = E[m.cell] + m.off * (E[m.cell + 1] - E[m.cell]);
        // Speed-limited kick and drift (Eqs. slpicEOMx, slpicEOMv).
        m.vx = kick(m, qmdt[s] * Ex, s);
        R s1 = m.vx * m.vx + m.vy * m.vy + m.vz * m.vz;
        R v1 = std::sqrt(s1);
        R b1 = beta(v1, s);
        m.off = m.off + b1 * (m.vx * dtdx);
        R fl = std::floor(m.off);
        m.cell += (int)fl;
        m.off = m.off - fl;
        if (m.off >= (R)1) {
          m.off = 0;
          m.cell += 1;
        }
        // Absorbing electrodes; the flux through each is the sum of w_j of
        // the markers that cross it (Eq. j).
        if (m.cell < 0) {
          t.n_abs[s][0]++;
          t.w_abs[s][0] += (double)m.wj;
          if (s == ION) {
            t.w_cath_ion += (double)m.wj;
            const R g = yield(m);
            if (!(m.id & GEN_BIT)) {
              t.w_cath_ion_gen0 += (double)m.wj;
              t.w_gain_gen0 += (double)(g * m.wj);
            }
            R u[4];
            draws(m.id, s_now, ION, 0, u);
            if (cfg.emit && u[0] < g) {
              Marker<R> e;
              e.cell = 0; e.off = 0; e.vx = 0; e.vy = 0; e.vz = 0;
              e.wj = m.wj;  // flux weight carried over to the emitted electron
              e.id = GEN_BIT;
              born_e_see.push_back(e);
              t.n_see++;
              t.w_see += (double)m.wj;
            }
          }
          continue;
        }
        if (m.cell >= N) {
          t.n_abs[s][1]++;
          t.w_abs[s][1] += (double)m.wj;
          continue;
        }
        if (s == ELECTRON) collide(m, s1, v1, s_now, t, born_e_ionz, born_i);
        survivors.push_back(m);
      }
      sp[s].swap(survivors);
    }
    // Append births: ionization electrons, then emitted electrons; ions.
    for (auto& m : born_e_ionz) {
      m.id = (m.id & GEN_BIT) | next_id[ELECTRON]++;
      sp[ELECTRON].push_back(m);
    }
    for (auto& m : born_e_see) {
      m.id = (m.id & GEN_BIT) | next_id[ELECTRON]++;
      sp[ELECTRON].push_back(m);
    }
    for (auto& m : born_i) {
      m.id = (m.id & GEN_BIT) | next_id[ION]++;
      sp[ION].push_back(m);
    }
    // Deposit every live marker with its density weight.
    for (int s = 0; s < 2; ++s) {
      std::fill(charge[s].begin(), charge[s].end(), 0);
      for (const auto& m : sp[s]) deposit_one(m, s, charge[s]);
    }
    if (cfg.field_mode == 1) solve_field();
    for (int s = 0; s < 2; ++s) {
      t.n_live[s] = (int64_t)sp[s].size();
      double w = 0;
      for (const auto& m : sp[s]) w += (double)m.wj;
      t.w_live[s] = w;
    }
    history.push_back(t);
    step++;
  }

  // Null-collision Monte-Carlo collision of one electron (Sec. III).
  void collide(Marker<R>& m, R s1, R v1, uint32_t s_now, oracle_tally& t,
               std::vector<Marker<R>>& born_e, std::vector<Marker<R>>& born_i) {
    if (!(collision_draw(m.id, s_now) < P0)) return;
    t.n_candidates++;
    R u[4];  // u[1]: process, u[2], u[3]: angles (u[0] unused)
    draws(m.id, s_now, ELECTRON, 0, u);
    R vb = v1 > vlim[ELECTRON] ? vlim[ELECTRON] : v1;  // beta v
    if (vb > vb_cap) {
      vb = vb_cap;
      t.n_majorant++;
    }
    R c = ndt * vb;
    R eps = s1 * K_E;
    R xs[5];
    xsec(eps, xs);
    R r = u[1] * P0;
    // the first process whose cumulative rate exceeds the draw: elastic,
    // excitation level 1..n_exc, ionization; none: a null collision
    int k = 0;
    while (k < n_proc && !(r < c * xs[k])) ++k;
    if (k == n_proc) return;
    const int proc = k == 0 ? 0 : (k <= n_exc ? 1 : 2);
    t.n_coll[proc]++;
    const R kv = K_V[ELECTRON];
    if (proc == 0) {
      // Elastic, Vahedi-Surendra: cos chi = (2 + eps - 2 (1 + eps)^u) / eps.
      // Both 1 - cos chi = 2 ((1 + eps)^u - 1) / eps and
      // 1 + cos chi = 2 (1 + eps) (1 - (1 + eps)^(u - 1)) / eps are formed
      // without cancellation (expm1 of u log1p(eps) and of -(1 - u) log1p(eps)),
      // so sin chi = sqrt((1 - cos chi)(1 + cos chi)) keeps its relative
      // precision for forward and backward scattering; recoil energy loss
      // eps 2 m/M (1 - cos chi).
      R L = std::log1p(eps);
      R em = std::expm1(u[2] * L);
      R ep = -std::expm1(-((R)1 - u[2]) * L);
      R omc = (em + em) / eps;
      R opc = (((R)1 + eps) * (ep + ep)) / eps;
      omc = std::min((R)2, std::max((R)0, omc));
      opc = std::min((R)2, std::max((R)0, opc));
      R cc = omc <= (R)1 ? (R)1 - omc : opc - (R)1;
      R sc = std::sqrt(omc * opc);
      R ph = two_pi * u[3];
      R cp = std::cos(ph), spn = std::sin(ph);
      R e_new = eps * ((R)1 - R2 * omc);
      R ux = m.vx / v1, uy = m.vy / v1, uz = m.vz / v1;
      rotate(ux, uy, uz, cc, sc, cp, spn);
      R v_new = std::sqrt(e_new * kv);
      m.vx = v_new * ux;
      m.vy = v_new * uy;
      m.vz = v_new * uz;
    } else if (proc == 1) {
      R e_new = eps - e_ex[k - 1];
      if (e_new < (R)0) {
        e_new = 0;
        t.n_clamp++;
      }
      isotropic(std::sqrt(e_new * kv), u[2], u[3], m.vx, m.vy, m.vz);
    } else {
      R e_av = eps - e_io;
      if (e_av < (R)0) {
        e_av = 0;
        t.n_clamp++;
      }
      t.w_ionz += (double)m.wj;
      R b[4];
      draws(m.id, s_now, ELECTRON, 1, b);
      R e_sec = b[0] * e_av;
      R e_pri = e_av - e_sec;
      isotropic(std::sqrt(e_pri * kv), u[2], u[3], m.vx, m.vy, m.vz);
      Marker<R> e;
      e.cell = m.cell;
      e.off = m.off;
      isotropic(std::sqrt(e_sec * kv), b[1], b[2], e.vx, e.vy, e.vz);
      e.wj = m.wj;
      e.id = m.id & GEN_BIT;
      born_e.push_back(e);
      // Ion at rest in the gas frame plus a Maxwellian at the gas
      // temperature (Box-Muller on a third block of draws).
      R g[4];
      draws(m.id, s_now, ELECTRON, 2, g);
      R r1 = std::sqrt((R)-2 * std::log(g[0]));
      R r2 = std::sqrt((R)-2 * std::log(g[2]));
      R a1 = two_pi * g[1], a2 = two_pi * g[3];
      Marker<R> ion;
      ion.cell = m.cell;
      ion.off = m.off;
      ion.vx = sigT_ion * (r1 * std::cos(a1));
      ion.vy = sigT_ion * (r1 * std::sin(a1));
      ion.vz = sigT_ion * (r2 * std::cos(a2));
      ion.wj = m.wj;
      ion.id = m.id & GEN_BIT;
      born_i.push_back(ion);
    }
  }

  // Initial markers.  mode 0: at the cathode, uniform in the first cell, given
  // energy, directions uniform on the forward (+x) hemisphere; mode 1: at the
  // cathode at rest; mode 2: uniform in the gap, energy log-uniform in
  // [e_lo, e_hi], isotropic; mode 3: uniform in the gap, Maxwellian at the gas
  // temperature.
  void seed(int s, int64_t n, int mode, double e0, double e_lo, double e_hi,
            double wj) {
    const R lr = (R)std::log(e_hi / e_lo);
    const R elo = (R)e_lo;
    const R ekin = (R)e0;
    const R Nr = (R)N;
    const R below1 = std::nextafter((R)1, (R)0);
    const R sigT = (R)std::sqrt(kKB * cfg.T_K / cfg.mass[s]);
    for (int64_t i = 0; i < n; ++i) {
      Marker<R> m;
      m.id = next_id[s]++;
      m.wj = (R)wj;
      R u[4];
      draws(m.id, SEED_STEP, s, 0, u);
      if (mode == 0 || mode == 1) {
        m.cell = 0;
        if (mode == 0) {
          m.off = u[0];
          R v = std::sqrt(ekin * K_V[s]);
          R ct = u[1];
          R st = std::sqrt(std::max((R)0, ((R)1 - ct) * ((R)1 + ct)));
          R ph = two_pi * u[2];
          m.vx = v * ct;
          m.vy = v * (st * std::cos(ph));
          m.vz = v * (st * std::sin(ph));
        } else {
          m.off = 0; m.vx = 0; m.vy = 0; m.vz = 0;
        }
      } else {
        R p = u[0] * Nr;
        R fl = std::floor(p);
        m.cell = (int)fl;
        m.off = p - fl;
        if (m.cell >= N) {
          m.cell = N - 1;
          m.off = below1;
        }
        if (mode == 2) {
          R e = elo * std::exp(u[1] * lr);
          isotropic(std::sqrt(e * K_V[s]), u[2], u[3], m.vx, m.vy, m.vz);
        } else {
          R g[4];
          draws(m.id, SEED_STEP, s, 1, g);
          R r1 = std::sqrt((R)-2 * std::log(u[1]));
          R r2 = std::sqrt((R)-2 * std::log(u[3]));
          R a1 = two_pi * u[2], a2 = two_pi * g[0];
          m.vx = sigT * (r1 * std::cos(a1));
          m.vy = sigT * (r1 * std::sin(a1));
          m.vz = sigT * (r2 * std::cos(a2));
        }
      }
      sp[s].push_back(m);
    }
  }

  void deposit_all() {
    for (int s = 0; s < 2; ++s) {
      std::fill(charge[s].begin(), charge[s].end(), 0);
      for (const auto& m : sp[s]) deposit_one(m, s, charge[s]);
    }
  }
};

struct Handle {
  int precision;
  Sim<double>* d = nullptr;
  Sim<float>* f = nullptr;
};

template <typename F>
void visit(Handle* h, F fn) {
  if (h->precision == 32) fn(*h->f);
  else fn(*h->d);
}

}  // namespace

extern "C" {

void oracle_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1,
                   uint32_t* out) {
  philox4x32_10(ctr, k0, k1, out);
}

void oracle_philox2_many(const uint32_t* ctr, int64_t n, uint32_t k, uint32_t* out) {
  for (int64_t i = 0; i < n; ++i) philox2x32_10(ctr + 2 * i, k, out + 2 * i);
}

// Many blocks at once: ctr is n x 4, out is n x 4.
void oracle_philox_many(const uint32_t* ctr, int64_t n, uint32_t k0,
                        uint32_t k1, uint32_t* out) {
  for (int64_t i = 0; i < n; ++i) philox4x32_10(ctr + 4 * i, k0, k1, out + 4 * i);
}

double oracle_uniform64(uint32_t x) { return uniform01<double>(x); }
float oracle_uniform32(uint32_t x) { return uniform01<float>(x); }

void* oracle_create(const oracle_config* c) {
  if (!c || c->n_cells < 1 || !(c->d > 0) || !(c->dt >= 0)) return nullptr;
  Handle* h = new Handle;
  h->precision = c->precision == 32 ? 32 : 64;
  if (h->precision == 32) {
    h->f = new Sim<float>;
    h->f->init(*c);
  } else {
    h->d = new Sim<double>;
    h->d->init(*c);
  }
  return h;
}

void oracle_destroy(void* hp) {
  Handle* h = (Handle*)hp;
  if (!h) return;
  delete h->d;
  delete h->f;
  delete h;
}

// Load n markers of species s from FP32 arrays (the storage format); in FP64
// mode they are widened exactly.  Replaces the species' markers.
int oracle_load(void* hp, int s, int64_t n, const int32_t* cell,
                const float* off, const float* vx, const float* vy,
                const float* vz, const float* wj, const uint32_t* id,
                uint32_t next_id) {
  Handle* h = (Handle*)hp;
  if (!h || s < 0 || s > 1 || n < 0) return -1;
  int bad = 0;
  visit(h, [&](auto& sim) {
    using R = decltype(sim.K_E);
    sim.sp[s].clear();
    for (int64_t i = 0; i < n; ++i) {
      Marker<R> m;
      m.cell = cell[i];
      m.off = (R)off[i];
      m.vx = (R)vx[i]; m.vy = (R)vy[i]; m.vz = (R)vz[i];
      m.wj = (R)wj[i];
      m.id = id[i];
      if (m.cell < 0 || m.cell >= sim.N || !(m.off >= 0) || !(m.off < 1)) bad = 1;
      sim.sp[s].push_back(m);
    }
    sim.next_id[s] = next_id;
  });
  return bad ? -2 : 0;
}

int oracle_seed(void* hp, int s, int64_t n, int mode, double e0, double e_lo,
                double e_hi, double wj) {
  Handle* h = (Handle*)hp;
  if (!h || s < 0 || s > 1 || n < 0 || mode < 0 || mode > 3) return -1;
  visit(h, [&](auto& sim) { sim.seed(s, n, mode, e0, e_lo, e_hi, wj); });
  return 0;
}

int oracle_step(void* hp, int64_t nsteps) {
  Handle* h = (Handle*)hp;
  if (!h || nsteps < 0) return -1;
  visit(h, [&](auto& sim) {
    for (int64_t i = 0; i < nsteps; ++i) sim.one_step();
  });
  return 0;
}

// The kick of n markers of species s (tests): new v_x for velocities
// (vx, vy, vz) and unlimited increments A, in the oracle's precision.
int oracle_kick(void* hp, int s, int64_t n, const double* vx, const double* vy,
                const double* vz, const double* A, double* out) {
  Handle* h = (Handle*)hp;
  if (!h || s < 0 || s > 1 || n < 0) return -1;
  visit(h, [&](auto& sim) {
    using R = decltype(sim.K_E);
    for (int64_t i = 0; i < n; ++i) {
      Marker<R> m;
      m.cell = 0; m.off = 0; m.wj = 1; m.id = 0;
      m.vx = (R)vx[i]; m.vy = (R)vy[i]; m.vz = (R)vz[i];
      out[i] = (double)sim.kick(m, (R)A[i], s);
    }
  });
  return 0;
}

// Deposit the current markers (no push), as the step's deposit would.
int oracle_deposit(void* hp) {
  Handle* h = (Handle*)hp;
  if (!h) return -1;
  visit(h, [&](auto& sim) { sim.deposit_all(); });
  return 0;
}

int oracle_solve_field(void* hp) {
  Handle* h = (Handle*)hp;
  if (!h) return -1;
  visit(h, [&](auto& sim) { sim.solve_field(); });
  return 0;
}

int64_t oracle_count(void* hp, int s) {
  Handle* h = (Handle*)hp;
  int64_t n = -1;
  if (!h || s < 0 || s > 1) return -1;
  visit(h, [&](auto& sim) { n = (int64_t)sim.sp[s].size(); });
  return n;
}

uint32_t oracle_next_id(void* hp, int s) {
  Handle* h = (Handle*)hp;
  uint32_t n = 0;
  visit(h, [&](auto& sim) { n = sim.next_id[s]; });
  return n;
}

int oracle_get(void* hp, int s, int32_t* cell, double* off, double* vx,
               double* vy, double* vz, double* wj, uint32_t* id) {
  Handle* h = (Handle*)hp;
  if (!h || s < 0 || s > 1) return -1;
  visit(h, [&](auto& sim) {
    for (size_t i = 0; i < sim.sp[s].size(); ++i) {
      const auto& m = sim.sp[s][i];
      cell[i] = m.cell;
      off[i] = (double)m.off;
      vx[i] = (double)m.vx; vy[i] = (double)m.vy; vz[i] = (double)m.vz;
      wj[i] = (double)m.wj;
      id[i] = m.id;
    }
  });
  return 0;
}

int oracle_charge(void* hp, int s, int64_t* out) {
  Handle* h = (Handle*)hp;
  if (!h || s < 0 || s > 1) return -1;
  visit(h, [&](auto& sim) {
    std::copy(sim.charge[s].begin(), sim.charge[s].end(), out);
  });
  return 0;
}

int oracle_field(void* hp, double* phi, double* E) {
  Handle* h = (Handle*)hp;
  if (!h) return -1;
  visit(h, [&](auto& sim) {
    std::copy(sim.phi.begin(), sim.phi.end(), phi);
    std::copy(sim.E64.begin(), sim.E64.end(), E);
  });
  return 0;
}

// Set the field at the nodes (used by tests that impose a field).
int oracle_set_field(void* hp, const double* E) {
  Handle* h = (Handle*)hp;
  if (!h) return -1;
  visit(h, [&](auto& sim) {
    using R = decltype(sim.K_E);
    for (int k = 0; k <= sim.N; ++k) {
      sim.E64[k] = E[k];
      sim.E[k] = (R)E[k];
    }
  });
  return 0;
}

int64_t oracle_history_len(void* hp) {
  Handle* h = (Handle*)hp;
  int64_t n = 0;
  visit(h, [&](auto& sim) { n = (int64_t)sim.history.size(); });
  return n;
}

int oracle_history(void* hp, oracle_tally* out) {
  Handle* h = (Handle*)hp;
  if (!h) return -1;
  visit(h, [&](auto& sim) {
    std::copy(sim.history.begin(), sim.history.end(), out);
  });
  return 0;
}

// The constants the step uses, as doubles, for tests: P0 (null-collision
// majorant probability), vb_cap, ndt.
int oracle_constants(void* hp, double* out3) {
  Handle* h = (Handle*)hp;
  if (!h) return -1;
  visit(h, [&](auto& sim) {
    out3[0] = (double)sim.P0;
    out3[1] = (double)sim.vb_cap;
    out3[2] = (double)sim.ndt;
  });
  return 0;
}

// Interpolated cumulative cross sections at energies eps[n] (tests): elastic,
// elastic plus every excitation level, total.
int oracle_xsec(void* hp, const double* eps, int64_t n, double* out) {
  Handle* h = (Handle*)hp;
  if (!h) return -1;
  visit(h, [&](auto& sim) {
    using R = decltype(sim.K_E);
    for (int64_t i = 0; i < n; ++i) {
      R xs[5];
      sim.xsec((R)eps[i], xs);
      out[3 * i] = (double)xs[0];
      out[3 * i + 1] = (double)xs[sim.n_exc];
      out[3 * i + 2] = (double)xs[sim.n_proc - 1];
    }
  });
  return 0;
}

// Time-step and run-length rules of the paper (Sec. IV): dt = dx / v0 with
// v0 = sqrt(2 e V / M) for SLPIC, dt = dx / vmax with vmax = sqrt(2 e V / m_e)
// for PIC; the classification window is 30 ion crossing times
// 30 sqrt(2 M d / (e E)), E = V / d.
double oracle_dt_slpic(double d, int cells, double V, double M) {
  return (d / cells) / std::sqrt(2.0 * kQe * V / M);
}
double oracle_dt_pic(double d, int cells, double V) {
  return (d / cells) / std::sqrt(2.0 * kQe * V / kMe);
}
double oracle_ion_crossing_time(double d, double V, double M) {
  double E = V / d;
  return std::sqrt(2.0 * M * d / (kQe * E));
}

}  // extern "C"
