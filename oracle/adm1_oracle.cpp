// CHAD ADM1 oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, FP64 CPU implementation of what the per-particle hot path
// computes.  Only the tests, the smoke check and the benchmark's CPU-baseline
// leg may load this library; the product path never does.  It shares no code,
// header or table with the CUDA library: the only common inputs are the
// parameter values and seeded populations produced by the input generator.
//
// What it follows (paper sections / equations):
//   * Sec. 2.2, Eq. 2     : per-particle CSTR mass balance
//                           dS_i/dt = D (S_in,i - S_i) + sum_j rho_j nu_ij,
//                           written here with an explicit Petersen matrix nu.
//   * Eq. 3-4 (reading)   : Hill pH inhibition in concentration form,
//                           I = K^n / (K^n + S_H^n), K = 10^-(LL+UL)/2,
//                           n = 3 / (UL - LL).
//   * Eq. 5-6             : non-competitive inhibition 1/(1 + S_I/K_I) and
//                           substrate limitation S/(S + K).
//   * Eq. 7               : charge balance E(S_H) = 0, solved by Newton with
//                           a bisection safeguard; S_H is algebraic.
//   * Sec. 2.3            : each AD particle is a CSTR of volume V/N; the gas
//                           share and k_p scale with V_p so the particle
//                           equations are intensive.
//   * Sec. 2.3 / 4.3      : particles are advected by the flow and integrated
//                           independently over each coupling interval;
//                           threads take equal chunks of particles.
//   * Integrator (reading): the paper names no scheme; this is the
//                           Rosenbrock 2(3) W-method of Shampine & Reichelt
//                           ("The MATLAB ODE Suite", 1997) with an embedded
//                           error estimate; J is computed by forward-mode
//                           automatic differentiation with dual numbers.
//   * Advection (reading) : Philox4x64-10 (Salmon et al., SC'11) drives an
//                           Irwin-Hall(12) Gaussian; rigid swirl rotation;
//                           reflecting cylinder walls.
//
// Parity pins: tests/test_oracle_pins.py and tests/test_oracle_pins_kinetics.py
// (tests/test_oracle_mutations.py checks that planted mistakes fail them).
// Absolute values against the
// paper's Fig. 3 / Table 3 are parity unpinned (the benchmark data is not
// available).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>
#include <algorithm>

namespace {

constexpr int NS = 29;
constexpr int NLIQ = 26;   // liquid states (rows of the Petersen matrix)
constexpr int NPROC = 22;  // 19 biochemical processes + 3 gas transfers

enum St {
  S_su, S_aa, S_fa, S_va, S_bu, S_pro, S_ac, S_h2, S_ch4, S_IC, S_IN, S_I,
  X_c, X_ch, X_pr, X_li, X_su, X_aa, X_fa, X_c4, X_pro, X_ac, X_h2, X_I,
  S_cat, S_an, G_h2, G_ch4, G_co2
};

// Parameter layout (must list the same names, in the same order, as the
// input generator; a test compares the lists).
#define ORACLE_PARAMS(X) \
  X(f_sI_xc) X(f_xI_xc) X(f_ch_xc) X(f_pr_xc) X(f_li_xc) \
  X(N_xc) X(N_I) X(N_aa) X(N_bac) \
  X(C_xc) X(C_sI) X(C_ch) X(C_pr) X(C_li) X(C_xI) X(C_su) X(C_aa) X(C_fa) \
  X(C_bu) X(C_pro) X(C_ac) X(C_bac) X(C_va) X(C_ch4) \
  X(f_fa_li) X(f_h2_su) X(f_bu_su) X(f_pro_su) X(f_ac_su) \
  X(f_h2_aa) X(f_va_aa) X(f_bu_aa) X(f_pro_aa) X(f_ac_aa) \
  X(f_ac_fa) X(f_h2_fa) X(f_pro_va) X(f_ac_va) X(f_h2_va) X(f_ac_bu) X(f_h2_bu) \
  X(f_ac_pro) X(f_h2_pro) \
  X(Y_su) X(Y_aa) X(Y_fa) X(Y_c4) X(Y_pro) X(Y_ac) X(Y_h2) \
  X(k_dis) X(k_hyd_ch) X(k_hyd_pr) X(k_hyd_li) \
  X(k_m_su) X(k_m_aa) X(k_m_fa) X(k_m_c4) X(k_m_pro) X(k_m_ac) X(k_m_h2) \
  X(k_dec_X_su) X(k_dec_X_aa) X(k_dec_X_fa) X(k_dec_X_c4) X(k_dec_X_pro) \
  X(k_dec_X_ac) X(k_dec_X_h2) \
  X(K_S_IN) X(K_S_su) X(K_S_aa) X(K_S_fa) X(K_S_c4) X(K_S_pro) X(K_S_ac) X(K_S_h2) \
  X(K_I_h2_fa) X(K_I_h2_c4) X(K_I_h2_pro) X(K_I_nh3) \
  X(pH_LL_aa) X(pH_UL_aa) X(pH_LL_ac) X(pH_UL_ac) X(pH_LL_h2) X(pH_UL_h2) \
  X(R) X(R_J) X(T_base) \
  X(pK_w) X(pK_a_va) X(pK_a_bu) X(pK_a_pro) X(pK_a_ac) X(pK_a_co2) X(pK_a_IN) \
  X(dH_K_w) X(dH_K_a_co2) X(dH_K_a_IN) \
  X(K_H_co2) X(K_H_ch4) X(K_H_h2) X(dH_K_H_co2) X(dH_K_H_ch4) X(dH_K_H_h2) \
  X(p_h2o_base) X(p_h2o_theta) \
  X(k_La) X(k_p) X(V_liq_ref) X(P_atm) \
  X(Ea_over_R) X(T_ref_kin)

enum Pi {
#define X(n) P_##n,
  ORACLE_PARAMS(X)
#undef X
  NPARAM
};
const char* kParamNames[] = {
#define X(n) #n,
  ORACLE_PARAMS(X)
#undef X
};

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual pow_n(Dual a, double n) {  // a^n for a > 0
  double p = std::pow(a.v, n);
  return Dual(p, n * std::pow(a.v, n - 1.0) * a.d);
}
inline double pow_n(double a, double n) { return std::pow(a, n); }
inline double val(double x) { return x; }
inline double val(Dual x) { return x.v; }

// ------------------------------------------------- per-particle model constants
struct Model {
  // temperature-scaled kinetic constants (1/d)
  double k_dis, k_hyd_ch, k_hyd_pr, k_hyd_li;
  double k_m_su, k_m_aa, k_m_fa, k_m_c4, k_m_pro, k_m_ac, k_m_h2, k_dec[7];
  double K_S_IN, K_S_su, K_S_aa, K_S_fa, K_S_c4, K_S_pro, K_S_ac, K_S_h2;
  double K_I_h2_fa, K_I_h2_c4, K_I_h2_pro, K_I_nh3;
  double K_pH_aa, n_aa, K_pH_ac, n_ac, K_pH_h2, n_h2;
  // acid-base and gas constants at T
  double K_w, K_a_va, K_a_bu, K_a_pro, K_a_ac, K_a_co2, K_a_IN;
  double K_H_co2, K_H_ch4, K_H_h2, p_h2o, RT, P_atm, k_La;
  double kp_over_Vgas;   // k_p,digester / V_gas  (1/(d bar))
  double Vliq_over_Vgas;
  double nu[NLIQ][NPROC];  // Petersen matrix, liquid rows
};

// Petersen matrix (Eq. 2): one column per process, one row per liquid state.
// Carbon (S_IC) and nitrogen (S_IN) coefficients of the biochemical processes
// are the closing terms -sum_i C_i nu_ij and -sum_i N_i nu_ij over the organic
// species, so C and N are conserved per process by construction.
void build_petersen(const double* p, double nu[NLIQ][NPROC]) {
  for (int i = 0; i < NLIQ; ++i)
    for (int j = 0; j < NPROC; ++j) nu[i][j] = 0.0;
  const double Ysu = p[P_Y_su], Yaa = p[P_Y_aa], Yfa = p[P_Y_fa], Yc4 = p[P_Y_c4];
  const double Ypro = p[P_Y_pro], Yac = p[P_Y_ac], Yh2 = p[P_Y_h2];
  // 1 disintegration of X_c
  nu[X_c][0] = -1.0;
  nu[S_I][0] = p[P_f_sI_xc];
  nu[X_ch][0] = p[P_f_ch_xc];
  nu[X_pr][0] = p[P_f_pr_xc];
  nu[X_li][0] = p[P_f_li_xc];
  nu[X_I][0] = p[P_f_xI_xc];
  // 2-4 hydrolysis
  nu[X_ch][1] = -1.0; nu[S_su][1] = 1.0;
  nu[X_pr][2] = -1.0; nu[S_aa][2] = 1.0;
  nu[X_li][3] = -1.0; nu[S_su][3] = 1.0 - p[P_f_fa_li]; nu[S_fa][3] = p[P_f_fa_li];
  // 5 uptake of sugars
  nu[S_su][4] = -1.0;
  nu[S_h2][4] = (1.0 - Ysu) * p[P_f_h2_su];
  nu[S_bu][4] = (1.0 - Ysu) * p[P_f_bu_su];
  nu[S_pro][4] = (1.0 - Ysu) * p[P_f_pro_su];
  nu[S_ac][4] = (1.0 - Ysu) * p[P_f_ac_su];
  nu[X_su][4] = Ysu;
  // 6 uptake of amino acids
  nu[S_aa][5] = -1.0;
  nu[S_h2][5] = (1.0 - Yaa) * p[P_f_h2_aa];
  nu[S_va][5] = (1.0 - Yaa) * p[P_f_va_aa];
  nu[S_bu][5] = (1.0 - Yaa) * p[P_f_bu_aa];
  nu[S_pro][5] = (1.0 - Yaa) * p[P_f_pro_aa];
  nu[S_ac][5] = (1.0 - Yaa) * p[P_f_ac_aa];
  nu[X_aa][5] = Yaa;
  // 7 uptake of LCFA
  nu[S_fa][6] = -1.0;
  nu[S_h2][6] = (1.0 - Yfa) * p[P_f_h2_fa];
  nu[S_ac][6] = (1.0 - Yfa) * p[P_f_ac_fa];
  nu[X_fa][6] = Yfa;
  // 8 uptake of valerate
  nu[S_va][7] = -1.0;
  nu[S_pro][7] = (1.0 - Yc4) * p[P_f_pro_va];
  nu[S_ac][7] = (1.0 - Yc4) * p[P_f_ac_va];
  nu[S_h2][7] = (1.0 - Yc4) * p[P_f_h2_va];
  nu[X_c4][7] = Yc4;
  // 9 uptake of butyrate
  nu[S_bu][8] = -1.0;
  nu[S_ac][8] = (1.0 - Yc4) * p[P_f_ac_bu];
  nu[S_h2][8] = (1.0 - Yc4) * p[P_f_h2_bu];
  nu[X_c4][8] = Yc4;
  // 10 uptake of propionate
  nu[S_pro][9] = -1.0;
  nu[S_ac][9] = (1.0 - Ypro) * p[P_f_ac_pro];
  nu[S_h2][9] = (1.0 - Ypro) * p[P_f_h2_pro];
  nu[X_pro][9] = Ypro;
  // 11 uptake of acetate
  nu[S_ac][10] = -1.0;
  nu[S_ch4][10] = 1.0 - Yac;
  nu[X_ac][10] = Yac;
  // 12 uptake of hydrogen
  nu[S_h2][11] = -1.0;
  nu[S_ch4][11] = 1.0 - Yh2;
  nu[X_h2][11] = Yh2;
  // 13-19 decay of the seven biomasses into X_c
  const int bio[7] = {X_su, X_aa, X_fa, X_c4, X_pro, X_ac, X_h2};
  for (int k = 0; k < 7; ++k) {
    nu[bio[k]][12 + k] = -1.0;
    nu[X_c][12 + k] = 1.0;
  }
  // carbon and nitrogen content of each liquid species (kmol per kgCOD)
  double C[NLIQ] = {0}, N[NLIQ] = {0};
  C[S_su] = p[P_C_su]; C[S_aa] = p[P_C_aa]; C[S_fa] = p[P_C_fa]; C[S_va] = p[P_C_va];
  C[S_bu] = p[P_C_bu]; C[S_pro] = p[P_C_pro]; C[S_ac] = p[P_C_ac]; C[S_ch4] = p[P_C_ch4];
  C[S_I] = p[P_C_sI]; C[X_c] = p[P_C_xc]; C[X_ch] = p[P_C_ch]; C[X_pr] = p[P_C_pr];
  C[X_li] = p[P_C_li]; C[X_I] = p[P_C_xI];
  for (int k = 0; k < 7; ++k) C[bio[k]] = p[P_C_bac];
  N[S_aa] = p[P_N_aa]; N[S_I] = p[P_N_I]; N[X_c] = p[P_N_xc]; N[X_pr] = p[P_N_aa];
  N[X_I] = p[P_N_I];
  for (int k = 0; k < 7; ++k) N[bio[k]] = p[P_N_bac];
  for (int j = 0; j < 19; ++j) {
    double sc = 0.0, sn = 0.0;
    for (int i = 0; i < NLIQ; ++i) {
      sc += C[i] * nu[i][j];
      sn += N[i] * nu[i][j];
    }
    nu[S_IC][j] = -sc;
    nu[S_IN][j] = -sn;
  }
  // 20-22 liquid-gas transfer of H2, CH4, CO2 (liquid side)
  nu[S_h2][19] = -1.0;
  nu[S_ch4][20] = -1.0;
  nu[S_IC][21] = -1.0;
}

// van 't Hoff factor exp(dH/R (1/T_base - 1/T))
double vant_hoff(const double* p, double dH, double T) {
  return std::exp(dH / p[P_R_J] * (1.0 / p[P_T_base] - 1.0 / T));
}

void make_model(const double* p, double T, double V_liq, double V_gas, Model& m) {
  const double arr = std::exp(-p[P_Ea_over_R] * (1.0 / T - 1.0 / p[P_T_ref_kin]));
  m.k_dis = p[P_k_dis] * arr;
  m.k_hyd_ch = p[P_k_hyd_ch] * arr;
  m.k_hyd_pr = p[P_k_hyd_pr] * arr;
  m.k_hyd_li = p[P_k_hyd_li] * arr;
  m.k_m_su = p[P_k_m_su] * arr;
  m.k_m_aa = p[P_k_m_aa] * arr;
  m.k_m_fa = p[P_k_m_fa] * arr;
  m.k_m_c4 = p[P_k_m_c4] * arr;
  m.k_m_pro = p[P_k_m_pro] * arr;
  m.k_m_ac = p[P_k_m_ac] * arr;
  m.k_m_h2 = p[P_k_m_h2] * arr;
  const Pi dec[7] = {P_k_dec_X_su, P_k_dec_X_aa, P_k_dec_X_fa, P_k_dec_X_c4,
                     P_k_dec_X_pro, P_k_dec_X_ac, P_k_dec_X_h2};
  for (int k = 0; k < 7; ++k) m.k_dec[k] = p[dec[k]] * arr;
  m.K_S_IN = p[P_K_S_IN]; m.K_S_su = p[P_K_S_su]; m.K_S_aa = p[P_K_S_aa];
  m.K_S_fa = p[P_K_S_fa]; m.K_S_c4 = p[P_K_S_c4]; m.K_S_pro = p[P_K_S_pro];
  m.K_S_ac = p[P_K_S_ac]; m.K_S_h2 = p[P_K_S_h2];
  m.K_I_h2_fa = p[P_K_I_h2_fa]; m.K_I_h2_c4 = p[P_K_I_h2_c4];
  m.K_I_h2_pro = p[P_K_I_h2_pro]; m.K_I_nh3 = p[P_K_I_nh3];
  m.K_pH_aa = std::pow(10.0, -(p[P_pH_LL_aa] + p[P_pH_UL_aa]) / 2.0);
  m.n_aa = 3.0 / (p[P_pH_UL_aa] - p[P_pH_LL_aa]);
  m.K_pH_ac = std::pow(10.0, -(p[P_pH_LL_ac] + p[P_pH_UL_ac]) / 2.0);
  m.n_ac = 3.0 / (p[P_pH_UL_ac] - p[P_pH_LL_ac]);
  m.K_pH_h2 = std::pow(10.0, -(p[P_pH_LL_h2] + p[P_pH_UL_h2]) / 2.0);
  m.n_h2 = 3.0 / (p[P_pH_UL_h2] - p[P_pH_LL_h2]);
  m.K_w = std::pow(10.0, -p[P_pK_w]) * vant_hoff(p, p[P_dH_K_w], T);
  m.K_a_va = std::pow(10.0, -p[P_pK_a_va]);
  m.K_a_bu = std::pow(10.0, -p[P_pK_a_bu]);
  m.K_a_pro = std::pow(10.0, -p[P_pK_a_pro]);
  m.K_a_ac = std::pow(10.0, -p[P_pK_a_ac]);
  m.K_a_co2 = std::pow(10.0, -p[P_pK_a_co2]) * vant_hoff(p, p[P_dH_K_a_co2], T);
  m.K_a_IN = std::pow(10.0, -p[P_pK_a_IN]) * vant_hoff(p, p[P_dH_K_a_IN], T);
  m.K_H_co2 = p[P_K_H_co2] * vant_hoff(p, p[P_dH_K_H_co2], T);
  m.K_H_ch4 = p[P_K_H_ch4] * vant_hoff(p, p[P_dH_K_H_ch4], T);
  m.K_H_h2 = p[P_K_H_h2] * vant_hoff(p, p[P_dH_K_H_h2], T);
  m.p_h2o = p[P_p_h2o_base] * std::exp(p[P_p_h2o_theta] * (1.0 / p[P_T_base] - 1.0 / T));
  m.RT = p[P_R] * T;
  m.P_atm = p[P_P_atm];
  m.k_La = p[P_k_La];
  // k_p is extensive (given for V_liq_ref); a digester of V_liq gets
  // k_p V_liq / V_liq_ref, and each particle the same ratio to its gas share.
  m.kp_over_Vgas = p[P_k_p] * (V_liq / p[P_V_liq_ref]) / V_gas;
  m.Vliq_over_Vgas = V_liq / V_gas;
  build_petersen(p, m.nu);
}

// ------------------------------------------------------- charge balance (Eq. 7)
// E(S_H) = S_cat + S_nh4 + S_H - S_hco3 - S_ac/64 - S_pro/112 - S_bu/160
//          - S_va/208 - K_w/S_H - S_an
template <class R>
R charge_residual(const Model& m, const R* y, R SH) {
  R S_nh3 = m.K_a_IN * y[S_IN] / (m.K_a_IN + SH);
  R S_nh4 = y[S_IN] - S_nh3;
  R S_hco3 = m.K_a_co2 * y[S_IC] / (m.K_a_co2 + SH);
  R S_ac_m = m.K_a_ac * y[S_ac] / (m.K_a_ac + SH);
  R S_pro_m = m.K_a_pro * y[S_pro] / (m.K_a_pro + SH);
  R S_bu_m = m.K_a_bu * y[S_bu] / (m.K_a_bu + SH);
  R S_va_m = m.K_a_va * y[S_va] / (m.K_a_va + SH);
  return y[S_cat] + S_nh4 + SH - S_hco3 - S_ac_m / 64.0 - S_pro_m / 112.0 -
         S_bu_m / 160.0 - S_va_m / 208.0 - m.K_w / SH - y[S_an];
}

// dE/dS_H by forward-mode AD
double charge_slope(const Model& m, const double* y, double SH) {
  Dual yd[NS];
  for (int i = 0; i < NS; ++i) yd[i] = Dual(y[i]);
  return charge_residual<Dual>(m, yd, Dual(SH, 1.0)).d;
}

struct NewtonStats {
  long iters = 0;
  long bisections = 0;
};

constexpr double SH_LO = 1e-14, SH_HI = 1.0;

// Bisection on the bracket [1e-14, 1] (geometric midpoint); E is strictly
// increasing in S_H so the root is unique.  Returns <= 0 if no sign change.
double charge_bisect(const Model& m, const double* y) {
  double lo = SH_LO, hi = SH_HI;
  double elo = charge_residual<double>(m, y, lo), ehi = charge_residual<double>(m, y, hi);
  if (!(elo < 0.0 && ehi > 0.0)) {
    if (elo == 0.0) return lo;
    if (ehi == 0.0) return hi;
    return -1.0;
  }
  for (int it = 0; it < 200; ++it) {
    double mid = std::sqrt(lo * hi);
    if (!(mid > lo && mid < hi)) break;
    double e = charge_residual<double>(m, y, mid);
    if (e == 0.0) return mid;
    if (e < 0.0) lo = mid; else hi = mid;
  }
  return std::sqrt(lo * hi);
}

// Newton on Eq. 7 from a guess; falls back to bisection when an iterate leaves
// (0, inf) or |E| stops decreasing.  Returns S_H (> 0) or -1 on failure.
double charge_solve(const Model& m, const double* y, double guess, NewtonStats* st,
                    int max_iters = 50) {
  double S = (guess > 0.0 && std::isfinite(guess)) ? guess : 1e-7;
  double prevE = INFINITY;
  for (int it = 0; it < max_iters; ++it) {
    double E = charge_residual<double>(m, y, S);
    if (st) st->iters++;
    if (!std::isfinite(E) || std::fabs(E) > std::fabs(prevE)) break;
    double dE = charge_slope(m, y, S);
    double dS = E / dE;
    double Sn = S - dS;
    if (!(Sn > 0.0) || !std::isfinite(Sn)) break;
    if (std::fabs(dS) <= 1e-14 * Sn || std::fabs(E) <= 1e-15) return Sn;
    prevE = E;
    S = Sn;
  }
  if (st) st->bisections++;
  return charge_bisect(m, y);
}

// ------------------------------------------------------- rates and f (Eq. 2-6)
template <class R>
void process_rates(const Model& m, const R* y, R SH, R* rho, R* q_over_Vgas) {
  // pH inhibition (Hill, concentration form)
  R I_pH_aa = pow_n(R(m.K_pH_aa), m.n_aa) / (pow_n(SH, m.n_aa) + pow_n(R(m.K_pH_aa), m.n_aa));
  R I_pH_ac = pow_n(R(m.K_pH_ac), m.n_ac) / (pow_n(SH, m.n_ac) + pow_n(R(m.K_pH_ac), m.n_ac));
  R I_pH_h2 = pow_n(R(m.K_pH_h2), m.n_h2) / (pow_n(SH, m.n_h2) + pow_n(R(m.K_pH_h2), m.n_h2));
  // inorganic nitrogen limitation (Eq. 6 form), hydrogen and ammonia inhibition (Eq. 5 form)
  R I_IN = R(1.0) / (R(1.0) + m.K_S_IN / y[S_IN]);
  R I_h2_fa = R(1.0) / (R(1.0) + y[S_h2] / m.K_I_h2_fa);
  R I_h2_c4 = R(1.0) / (R(1.0) + y[S_h2] / m.K_I_h2_c4);
  R I_h2_pro = R(1.0) / (R(1.0) + y[S_h2] / m.K_I_h2_pro);
  R S_nh3 = m.K_a_IN * y[S_IN] / (m.K_a_IN + SH);
  R I_nh3 = R(1.0) / (R(1.0) + S_nh3 / m.K_I_nh3);
  R I5 = I_pH_aa * I_IN;
  R I7 = I_pH_aa * I_IN * I_h2_fa;
  R I8 = I_pH_aa * I_IN * I_h2_c4;
  R I10 = I_pH_aa * I_IN * I_h2_pro;
  R I11 = I_pH_ac * I_IN * I_nh3;
  R I12 = I_pH_h2 * I_IN;

  rho[0] = m.k_dis * y[X_c];
  rho[1] = m.k_hyd_ch * y[X_ch];
  rho[2] = m.k_hyd_pr * y[X_pr];
  rho[3] = m.k_hyd_li * y[X_li];
  rho[4] = m.k_m_su * y[S_su] / (m.K_S_su + y[S_su]) * y[X_su] * I5;
  rho[5] = m.k_m_aa * y[S_aa] / (m.K_S_aa + y[S_aa]) * y[X_aa] * I5;
  rho[6] = m.k_m_fa * y[S_fa] / (m.K_S_fa + y[S_fa]) * y[X_fa] * I7;
  rho[7] = m.k_m_c4 * y[S_va] / (m.K_S_c4 + y[S_va]) * y[X_c4] *
           (y[S_va] / (y[S_bu] + y[S_va] + 1e-6)) * I8;
  rho[8] = m.k_m_c4 * y[S_bu] / (m.K_S_c4 + y[S_bu]) * y[X_c4] *
           (y[S_bu] / (y[S_bu] + y[S_va] + 1e-6)) * I8;
  rho[9] = m.k_m_pro * y[S_pro] / (m.K_S_pro + y[S_pro]) * y[X_pro] * I10;
  rho[10] = m.k_m_ac * y[S_ac] / (m.K_S_ac + y[S_ac]) * y[X_ac] * I11;
  rho[11] = m.k_m_h2 * y[S_h2] / (m.K_S_h2 + y[S_h2]) * y[X_h2] * I12;
  const int bio[7] = {X_su, X_aa, X_fa, X_c4, X_pro, X_ac, X_h2};
  for (int k = 0; k < 7; ++k) rho[12 + k] = m.k_dec[k] * y[bio[k]];

  // gas phase: partial pressures (bar), total pressure, gas outflow
  R p_h2 = y[G_h2] * m.RT / 16.0;
  R p_ch4 = y[G_ch4] * m.RT / 64.0;
  R p_co2 = y[G_co2] * m.RT;
  R P_gas = p_h2 + p_ch4 + p_co2 + m.p_h2o;
  *q_over_Vgas = m.kp_over_Vgas * (P_gas - m.P_atm) * P_gas / m.P_atm;
  // liquid-gas transfer
  R S_hco3 = m.K_a_co2 * y[S_IC] / (m.K_a_co2 + SH);
  R S_co2 = y[S_IC] - S_hco3;
  rho[19] = m.k_La * (y[S_h2] - 16.0 * m.K_H_h2 * p_h2);
  rho[20] = m.k_La * (y[S_ch4] - 64.0 * m.K_H_ch4 * p_ch4);
  rho[21] = m.k_La * (S_co2 - m.K_H_co2 * p_co2);
}

template <class R>
void rhs_given_SH(const Model& m, const double* y_in, double D, const R* y, R SH, R* f,
                  R* rho_out = nullptr) {
  R rho[NPROC], qv;
  process_rates<R>(m, y, SH, rho, &qv);
  for (int i = 0; i < NLIQ; ++i) {
    R acc = D * (y_in[i] - y[i]);
    for (int j = 0; j < NPROC; ++j)
      if (m.nu[i][j] != 0.0) acc += m.nu[i][j] * rho[j];
    f[i] = acc;
  }
  f[G_h2] = -y[G_h2] * qv + rho[19] * m.Vliq_over_Vgas;
  f[G_ch4] = -y[G_ch4] * qv + rho[20] * m.Vliq_over_Vgas;
  f[G_co2] = -y[G_co2] * qv + rho[21] * m.Vliq_over_Vgas;
  if (rho_out)
    for (int j = 0; j < NPROC; ++j) rho_out[j] = rho[j];
}

struct Particle {
  const Model* m;
  const double* y_in;
  double D;
  double SH;  // running S_H (Newton guess and last root)
  NewtonStats ns;
  bool newton_failed = false;
  bool h2_alg = false;  // S_h2 algebraic (Eq. 8) instead of differential
  double SH2 = 0.0;     // running S_h2 root (Newton guess and last root)
  Particle(const Model* m_, const double* y_in_, double D_, double SH_)
      : m(m_), y_in(y_in_), D(D_), SH(SH_) {}
};

// Eq. 8: E(S_h2) = the S_h2 mass balance (inflow - outflow + production -
// uptake - transfer to the gas) at y with S_h2 replaced by S, and dE/dS.
// E is strictly decreasing in S: uptake and transfer grow with S, while the
// hydrogen-inhibited producers and the outflow shrink.
double h2_residual(Particle& P, const double* y, double SH, double S, double* dE) {
  Dual yd[NS], f[NS];
  for (int i = 0; i < NS; ++i) yd[i] = Dual(y[i]);
  yd[S_h2] = Dual(S, 1.0);
  rhs_given_SH<Dual>(*P.m, P.y_in, P.D, yd, Dual(SH), f);
  if (dE) *dE = f[S_h2].d;
  return f[S_h2].v;
}

// Root of Eq. 8: Newton from the guess (stop at |dS| <= 1e-14 S), with a
// bisection fallback on a bracket [0, hi] grown by doubling from the guess.
double h2_solve(Particle& P, const double* y, double SH, double guess) {
  double S = (guess > 0.0 && std::isfinite(guess)) ? guess : 1e-8;
  double prevE = INFINITY;
  for (int it = 0; it < 50; ++it) {
    double dE;
    const double E = h2_residual(P, y, SH, S, &dE);
    P.ns.iters++;
    if (!std::isfinite(E) || std::fabs(E) > std::fabs(prevE) || !(dE < 0.0)) break;
    const double dS = E / dE;
    const double Sn = S - dS;
    if (!(Sn > 0.0) || !std::isfinite(Sn)) break;
    if (std::fabs(dS) <= 1e-14 * Sn || E == 0.0) return Sn;
    prevE = E;
    S = Sn;
  }
  P.ns.bisections++;
  double lo = 0.0, hi = std::max(guess > 0.0 ? guess : 0.0, 1e-12);
  for (int k = 0; k < 200 && h2_residual(P, y, SH, hi, nullptr) > 0.0; ++k) hi *= 2.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (h2_residual(P, y, SH, mid, nullptr) > 0.0) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

// f(y): solves Eq. 7 for S_H (warm start from the particle's running S_H);
// with S_h2 algebraic also Eq. 8 for S_h2, whose rate is then zero.
void rhs(Particle& P, const double* y, double* f) {
  double SH = charge_solve(*P.m, y, P.SH, &P.ns);
  if (!(SH > 0.0)) { P.newton_failed = true; SH = P.SH; }
  P.SH = SH;
  if (!P.h2_alg) {
    rhs_given_SH<double>(*P.m, P.y_in, P.D, y, SH, f);
    return;
  }
  double yy[NS];
  for (int i = 0; i < NS; ++i) yy[i] = y[i];
  P.SH2 = h2_solve(P, y, SH, P.SH2);
  yy[S_h2] = P.SH2;
  rhs_given_SH<double>(*P.m, P.y_in, P.D, yy, SH, f);
  f[S_h2] = 0.0;
}

// J = df/dy with S_H(y) differentiated through Eq. 7 (implicit function theorem)
// and, with S_h2 algebraic, S_h2(y) through Eq. 8: the S_h2 row and column
// are zero (the rate is zero and the stored S_h2 is only a guess).
void jacobian(Particle& P, const double* y, double* J /* NS x NS row-major */) {
  double SH = charge_solve(*P.m, y, P.SH, &P.ns);
  if (!(SH > 0.0)) { P.newton_failed = true; SH = P.SH; }
  P.SH = SH;
  const double dEdS = charge_slope(*P.m, y, SH);
  if (P.h2_alg) {
    P.SH2 = h2_solve(P, y, SH, P.SH2);
    double dE2;
    h2_residual(P, y, SH, P.SH2, &dE2);
    for (int k = 0; k < NS; ++k) {
      Dual yd[NS], f[NS];
      for (int i = 0; i < NS; ++i) yd[i] = Dual(y[i], (i == k && k != S_h2) ? 1.0 : 0.0);
      yd[S_h2] = Dual(P.SH2);
      const double dEdy = charge_residual<Dual>(*P.m, yd, Dual(SH)).d;
      const Dual SHd(SH, -dEdy / dEdS);
      rhs_given_SH<Dual>(*P.m, P.y_in, P.D, yd, SHd, f);  // dE2/dy_k at fixed S_h2
      yd[S_h2] = Dual(P.SH2, -f[S_h2].d / dE2);
      rhs_given_SH<Dual>(*P.m, P.y_in, P.D, yd, SHd, f);
      for (int i = 0; i < NS; ++i) J[i * NS + k] = (i == S_h2) ? 0.0 : f[i].d;
    }
    return;
  }
  for (int k = 0; k < NS; ++k) {
    Dual yd[NS];
    for (int i = 0; i < NS; ++i) yd[i] = Dual(y[i], i == k ? 1.0 : 0.0);
    const double dEdy = charge_residual<Dual>(*P.m, yd, Dual(SH)).d;
    const Dual SHd(SH, -dEdy / dEdS);
    Dual f[NS];
    rhs_given_SH<Dual>(*P.m, P.y_in, P.D, yd, SHd, f);
    for (int i = 0; i < NS; ++i) J[i * NS + k] = f[i].d;
  }
}

// ------------------------------------------------------- dense LU (textbook)
// Gaussian elimination with partial pivoting; ties go to the lowest row.
bool lu_factor(double* A, int* piv) {
  for (int k = 0; k < NS; ++k) {
    int p = k;
    double best = std::fabs(A[k * NS + k]);
    for (int i = k + 1; i < NS; ++i) {
      double v = std::fabs(A[i * NS + k]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (best == 0.0 || !std::isfinite(best)) return false;
    if (p != k)
      for (int j = 0; j < NS; ++j) std::swap(A[k * NS + j], A[p * NS + j]);
    for (int i = k + 1; i < NS; ++i) {
      A[i * NS + k] /= A[k * NS + k];
      for (int j = k + 1; j < NS; ++j) A[i * NS + j] -= A[i * NS + k] * A[k * NS + j];
    }
  }
  return true;
}

void lu_solve(const double* LU, const int* piv, double* b) {
  for (int k = 0; k < NS; ++k)
    if (piv[k] != k) std::swap(b[k], b[piv[k]]);
  for (int i = 1; i < NS; ++i)
    for (int j = 0; j < i; ++j) b[i] -= LU[i * NS + j] * b[j];
  for (int i = NS - 1; i >= 0; --i) {
    for (int j = i + 1; j < NS; ++j) b[i] -= LU[i * NS + j] * b[j];
    b[i] /= LU[i * NS + i];
  }
}

// ------------------------------------------------------- Rosenbrock 2(3) step
// Shampine & Reichelt (1997): d = 1/(2+sqrt 2), e32 = 6+sqrt 2, W = I - h d J,
//   k1 = W^-1 F0,  F1 = f(y + h/2 k1),  k2 = W^-1 (F1 - k1) + k1,
//   y1 = y + h k2, F2 = f(y1),  k3 = W^-1 (F2 - e32 (k2 - F1) - 2 (k1 - F0)),
//   err = h/6 (k1 - 2 k2 + k3).
const double RB_D = 1.0 / (2.0 + std::sqrt(2.0));
const double RB_E32 = 6.0 + std::sqrt(2.0);

enum Status { ST_OK = 0, ST_NEWTON = 1, ST_STEPS = 2, ST_HMIN = 4, ST_NEG = 8, ST_NAN = 16 };

struct StepStats {
  long accepted = 0, rejected = 0, newton_iters = 0, bisections = 0, lu_fail = 0;
};

// One step of size h from y with F0 = f(y) and J given.  Writes y1 and err.
bool rb_step(Particle& P, const double* y, const double* F0, const double* J, double h,
             double* y1, double* err) {
  double W[NS * NS];
  int piv[NS];
  for (int i = 0; i < NS; ++i)
    for (int j = 0; j < NS; ++j) W[i * NS + j] = (i == j ? 1.0 : 0.0) - h * RB_D * J[i * NS + j];
  if (!lu_factor(W, piv)) return false;
  double k1[NS], k2[NS], k3[NS], F1[NS], F2[NS], tmp[NS];
  for (int i = 0; i < NS; ++i) k1[i] = F0[i];
  lu_solve(W, piv, k1);
  for (int i = 0; i < NS; ++i) tmp[i] = y[i] + 0.5 * h * k1[i];
  rhs(P, tmp, F1);
  for (int i = 0; i < NS; ++i) k2[i] = F1[i] - k1[i];
  lu_solve(W, piv, k2);
  for (int i = 0; i < NS; ++i) k2[i] += k1[i];
  for (int i = 0; i < NS; ++i) y1[i] = y[i] + h * k2[i];
  rhs(P, y1, F2);
  for (int i = 0; i < NS; ++i) k3[i] = F2[i] - RB_E32 * (k2[i] - F1[i]) - 2.0 * (k1[i] - F0[i]);
  lu_solve(W, piv, k3);
  for (int i = 0; i < NS; ++i) err[i] = h / 6.0 * (k1[i] - 2.0 * k2[i] + k3[i]);
  return true;
}

constexpr double H_MIN = 1e-12;      // days
constexpr double H_DEFAULT = 1e-6;   // days, used when no previous step size exists

// Integrate one particle over [0, T_end] days.  fixed_n > 0 takes fixed_n
// equal steps without error control; otherwise the step controller runs.
int integrate_interval(Particle& P, double* y, double* h_io, double T_end, double rtol,
                       const double* atol, long max_steps, int fixed_n, StepStats& st) {
  int status = 0;
  double F0[NS], J[NS * NS], y1[NS], err[NS];
  if (fixed_n > 0) {
    const double h = T_end / fixed_n;
    for (int s = 0; s < fixed_n; ++s) {
      rhs(P, y, F0);
      jacobian(P, y, J);
      if (!rb_step(P, y, F0, J, h, y1, err)) { st.lu_fail++; status |= ST_NAN; break; }
      for (int i = 0; i < NS; ++i) y[i] = y1[i];
      if (P.h2_alg) y[S_h2] = P.SH2;  // root at y1 (the last evaluation of the step)
      st.accepted++;
    }
  } else {
    double t = 0.0;
    double h = (*h_io > 0.0 && std::isfinite(*h_io)) ? *h_io : H_DEFAULT;
    bool have_fj = false, rejected_prev = false;
    long steps = 0;
    while (t < T_end) {
      if (steps >= max_steps) { status |= ST_STEPS; break; }
      ++steps;
      double hh = h;
      bool last = false;
      if (hh >= (T_end - t) * (1.0 - 1e-12)) { hh = T_end - t; last = true; }
      if (!have_fj) {
        rhs(P, y, F0);
        jacobian(P, y, J);
        have_fj = true;
      }
      double norm;
      bool ok = rb_step(P, y, F0, J, hh, y1, err);
      if (!ok) { st.lu_fail++; norm = INFINITY; }
      else {
        norm = 0.0;
        for (int i = 0; i < NS; ++i) {
          double sc = atol[i] + rtol * std::max(std::fabs(y[i]), std::fabs(y1[i]));
          double e = std::fabs(err[i]) / sc;
          if (!(e <= norm)) norm = e;  // NaN propagates
        }
      }
      if (norm <= 1.0) {
        for (int i = 0; i < NS; ++i) y[i] = y1[i];
        if (P.h2_alg) y[S_h2] = P.SH2;  // root at y1 (the last evaluation of the step)
        t = last ? T_end : t + hh;
        have_fj = false;
        st.accepted++;
        double fac = (norm == 0.0) ? 5.0 : std::min(5.0, std::max(0.2, 0.8 * std::pow(norm, -1.0 / 3.0)));
        if (rejected_prev) fac = std::min(fac, 1.0);
        h = hh * fac;
        rejected_prev = false;
      } else {
        st.rejected++;
        double fac = std::isfinite(norm) ? std::max(0.2, 0.8 * std::pow(norm, -1.0 / 3.0)) : 0.2;
        h = hh * fac;
        rejected_prev = true;
        if (h < H_MIN) { status |= ST_HMIN; break; }
      }
    }
    *h_io = h;
  }
  if (P.newton_failed) status |= ST_NEWTON;
  for (int i = 0; i < NS; ++i) {
    if (!std::isfinite(y[i])) { status |= ST_NAN; break; }
  }
  for (int i = 0; i < NS; ++i)
    if (y[i] < -atol[i]) { status |= ST_NEG; break; }
  return status;
}

// ------------------------------------------------------- Philox4x64-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): 10 rounds of the 4x64 Philox S-box with Weyl-sequence key updates.
void philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    unsigned __int128 p0 = (unsigned __int128)M0 * c0;
    unsigned __int128 p1 = (unsigned __int128)M1 * c2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t n0 = hi1 ^ c1 ^ k0;
    uint64_t n1 = lo1;
    uint64_t n2 = hi0 ^ c3 ^ k1;
    uint64_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Standard-normal draw: Irwin-Hall sum of 12 uniforms (u = (b + 1/2) / 2^16
// for the 16-bit chunks b of one Philox block) minus 6.  Integer sum, one
// exact scaling: bit-identical on every IEEE machine.
double gauss_irwin_hall(uint64_t seed, uint64_t pid, uint64_t interval, uint64_t sub, uint64_t axis) {
  const uint64_t ctr[4] = {interval, sub, axis, 0};
  const uint64_t key[2] = {seed, pid};
  uint64_t w[4];
  philox4x64_10(ctr, key, w);
  uint64_t s = 0;
  for (int k = 0; k < 12; ++k) s += (w[k / 4] >> (16 * (k % 4))) & 0xFFFFULL;
  return ((double)s + 6.0) / 65536.0 - 6.0;
}

struct Flow {
  bool on;
  double U, R, H, sigma, slab_zmin, q_in;
  const double* y_in;
  uint64_t seed;
};

// Advance one particle's position over n_sub sub-steps of length dsub (s):
// rigid rotation by the angle U/R*dsub (cos/sin given), Gaussian displacement
// sigma*dsub*g per axis, reflection at r = R, z = 0 and z = H.
void advect_one(const Flow& fl, double c, double s, int n_sub, double dsub, uint64_t pid,
                uint64_t interval, double& x, double& y, double& z) {
  const double amp = fl.sigma * dsub;
  for (int k = 0; k < n_sub; ++k) {
    double xr = c * x - s * y;
    double yr = s * x + c * y;
    x = xr + amp * gauss_irwin_hall(fl.seed, pid, interval, (uint64_t)k, 0);
    y = yr + amp * gauss_irwin_hall(fl.seed, pid, interval, (uint64_t)k, 1);
    z = z + amp * gauss_irwin_hall(fl.seed, pid, interval, (uint64_t)k, 2);
    double r = std::sqrt(x * x + y * y);
    if (r > fl.R) {
      double g = (2.0 * fl.R - r) / r;
      x = x * g;
      y = y * g;
    }
    if (z < 0.0) z = -z;
    if (z > fl.H) z = 2.0 * fl.H - z;
  }
}

template <class F>
void parallel_chunks(long n, int n_threads, F fn) {
  if (n_threads <= 1 || n < 2) { fn(0L, n); return; }
  std::vector<std::thread> th;
  long chunk = (n + n_threads - 1) / n_threads;
  for (int t = 0; t < n_threads; ++t) {
    long a = t * chunk, b = std::min(n, a + chunk);
    if (a >= b) break;
    th.emplace_back([=]() { fn(a, b); });
  }
  for (auto& x : th) x.join();
}

}  // namespace

// =========================================================================
// C entry points (ctypes)
// =========================================================================
// ------------------------------------------------------- diffusion between particles
// SPH discretisation of the diffusion equation (Cleary & Monaghan, J. Comput.
// Phys. 148 (1999)) for particles of equal volume V, with the Wendland C2
// kernel of smoothing length h (support 2h) in the form of Eq. 1:
//   dC_i/dt = sum_{j != i} 2 D V (C_i - C_j) r_ij W'(r_ij) / (r_ij^2 + 0.01 h^2),
// pairwise antisymmetric, so the total of every species is conserved.  The
// soluble species (S_su .. S_I) and the lumped ions S_cat, S_an diffuse;
// particulates and the gas states do not.  Brute force over all pairs.
constexpr int N_DIFF = 14;
const int DIFF_STATES[N_DIFF] = {S_su, S_aa, S_fa, S_va, S_bu, S_pro, S_ac,
                                 S_h2, S_ch4, S_IC, S_IN, S_I, S_cat, S_an};

double wendland_dwdr(double r, double h) {
  const double q = r / h;
  if (q >= 2.0) return 0.0;
  const double alpha = 21.0 / (16.0 * M_PI * h * h * h);
  const double t = 1.0 - 0.5 * q;
  return -5.0 * alpha * q * t * t * t / h;
}

extern "C" {

int oracle_n_params(void) { return NPARAM; }
const char* oracle_param_name(int i) { return (i >= 0 && i < NPARAM) ? kParamNames[i] : nullptr; }
int oracle_n_states(void) { return NS; }
int oracle_n_processes(void) { return NPROC; }

// Petersen matrix of a parameter vector (NLIQ x NPROC row-major)
void oracle_petersen(const double* params, double* nu_out) {
  double nu[NLIQ][NPROC];
  build_petersen(params, nu);
  for (int i = 0; i < NLIQ; ++i)
    for (int j = 0; j < NPROC; ++j) nu_out[i * NPROC + j] = nu[i][j];
}

// Temperature-dependent constants: K_w, K_a_co2, K_a_IN, K_H_co2, K_H_ch4, K_H_h2, p_h2o, Arrhenius factor
void oracle_constants(const double* params, double T, double* out8) {
  Model m;
  make_model(params, T, 1.0, 1.0, m);
  out8[0] = m.K_w; out8[1] = m.K_a_co2; out8[2] = m.K_a_IN; out8[3] = m.K_H_co2;
  out8[4] = m.K_H_ch4; out8[5] = m.K_H_h2; out8[6] = m.p_h2o;
  out8[7] = m.k_dis / params[P_k_dis];
}

double oracle_charge_residual(const double* params, double T, const double* y, double SH) {
  Model m;
  make_model(params, T, 1.0, 1.0, m);
  return charge_residual<double>(m, y, SH);
}

// Newton with bisection fallback; returns S_H (<= 0 on failure)
double oracle_charge_solve(const double* params, double T, const double* y, double guess,
                           int max_iters, long* iters, long* bisections) {
  Model m;
  make_model(params, T, 1.0, 1.0, m);
  NewtonStats st;
  double r = charge_solve(m, y, guess, &st, max_iters);
  if (iters) *iters = st.iters;
  if (bisections) *bisections = st.bisections;
  return r;
}

double oracle_charge_bisect(const double* params, double T, const double* y) {
  Model m;
  make_model(params, T, 1.0, 1.0, m);
  return charge_bisect(m, y);
}

// f(y), S_H and the 22 process rates
int oracle_rhs(const double* params, double T, double V_liq, double V_gas, double D,
               const double* y_in, const double* y, double SH_guess, double* f_out,
               double* SH_out, double* rho_out) {
  Model m;
  make_model(params, T, V_liq, V_gas, m);
  NewtonStats st;
  double SH = charge_solve(m, y, SH_guess, &st);
  if (!(SH > 0.0)) return ST_NEWTON;
  double rho[NPROC];
  rhs_given_SH<double>(m, y_in, D, y, SH, f_out, rho);
  if (SH_out) *SH_out = SH;
  if (rho_out)
    for (int j = 0; j < NPROC; ++j) rho_out[j] = rho[j];
  return 0;
}

// f(y) with S_H given (no Newton)
void oracle_rhs_at(const double* params, double T, double V_liq, double V_gas, double D,
                   const double* y_in, const double* y, double SH, double* f_out) {
  Model m;
  make_model(params, T, V_liq, V_gas, m);
  rhs_given_SH<double>(m, y_in, D, y, SH, f_out);
}

// the 22 process rates with S_H given (no Newton); q_gas/V_gas in rho_out[22]
void oracle_rates_at(const double* params, double T, double V_liq, double V_gas,
                     const double* y, double SH, double* rho_out) {
  Model m;
  make_model(params, T, V_liq, V_gas, m);
  double qv;
  process_rates<double>(m, y, SH, rho_out, &qv);
  rho_out[NPROC] = qv;
}

// J = df/dy (forward-mode AD through the charge balance), NS x NS row-major
int oracle_jacobian(const double* params, double T, double V_liq, double V_gas, double D,
                    const double* y_in, const double* y, double SH_guess, double* J_out) {
  Model m;
  make_model(params, T, V_liq, V_gas, m);
  Particle P{&m, y_in, D, SH_guess};
  jacobian(P, y, J_out);
  return P.newton_failed ? ST_NEWTON : 0;
}

// f(y) with S_h2 algebraic (Eq. 8): S_H and S_h2 roots, f with a zero S_h2 rate
int oracle_rhs_h2alg(const double* params, double T, double V_liq, double V_gas, double D,
                     const double* y_in, const double* y, double SH_guess, double* f_out,
                     double* SH_out, double* SH2_out) {
  Model m;
  make_model(params, T, V_liq, V_gas, m);
  Particle P{&m, y_in, D, SH_guess};
  P.h2_alg = true;
  P.SH2 = y[S_h2];
  rhs(P, y, f_out);
  *SH_out = P.SH;
  *SH2_out = P.SH2;
  return P.newton_failed ? ST_NEWTON : 0;
}

// J = df/dy with S_h2 algebraic (Eq. 8), NS x NS row-major
int oracle_jacobian_h2alg(const double* params, double T, double V_liq, double V_gas, double D,
                          const double* y_in, const double* y, double SH_guess, double* J_out) {
  Model m;
  make_model(params, T, V_liq, V_gas, m);
  Particle P{&m, y_in, D, SH_guess};
  P.h2_alg = true;
  P.SH2 = y[S_h2];
  jacobian(P, y, J_out);
  return P.newton_failed ? ST_NEWTON : 0;
}

// One particle over dt_days.  stats: accepted, rejected, newton iterations, bisections.
int oracle_integrate(const double* params, double T, double V_liq, double V_gas, double D,
                     const double* y_in, double* y, double* SH, double* h, double dt_days,
                     double rtol, const double* atol, long max_steps, int fixed_n,
                     long* stats4, int h2_alg) {
  Model m;
  make_model(params, T, V_liq, V_gas, m);
  Particle P{&m, y_in, D, *SH};
  P.h2_alg = h2_alg != 0;
  P.SH2 = y[S_h2];
  StepStats st;
  int status = integrate_interval(P, y, h, dt_days, rtol, atol, max_steps, fixed_n, st);
  *SH = P.SH;
  if (stats4) {
    stats4[0] = st.accepted; stats4[1] = st.rejected;
    stats4[2] = P.ns.iters; stats4[3] = P.ns.bisections;
  }
  return status;
}

// n_sub explicit Euler steps of the SPH diffusion equation over dt_s seconds
// for the particles [a, b) of arrays of leading dimension ld: pos [3][ld] (m),
// y [NS][ld] in place.
void diffuse_range(long ld, long a, long b, const double* pos, double* y, double V, double D,
                   double h, double dt_s, int n_sub) {
  const long n = b - a;
  const double dt = dt_s / n_sub;
  std::vector<double> flux((size_t)N_DIFF * n);
  for (int sub = 0; sub < n_sub; ++sub) {
    for (long i = a; i < b; ++i) {
      double acc[N_DIFF] = {0};
      for (long j = a; j < b; ++j) {
        if (j == i) continue;
        const double dx = pos[i] - pos[j], dy = pos[ld + i] - pos[ld + j];
        const double dz = pos[2 * ld + i] - pos[2 * ld + j];
        const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
        if (r >= 2.0 * h) continue;
        const double wgt = 2.0 * D * V * r * wendland_dwdr(r, h) / (r * r + 0.01 * h * h);
        for (int k = 0; k < N_DIFF; ++k) {
          const int st = DIFF_STATES[k];
          acc[k] += wgt * (y[(long)st * ld + i] - y[(long)st * ld + j]);
        }
      }
      for (int k = 0; k < N_DIFF; ++k) flux[(size_t)k * n + (i - a)] = acc[k];
    }
    for (int k = 0; k < N_DIFF; ++k)
      for (long i = a; i < b; ++i)
        y[(long)DIFF_STATES[k] * ld + i] += dt * flux[(size_t)k * n + (i - a)];
  }
}

// Largest row sum max_i sum_j |w_ij| of the discrete diffusion operator over
// the particles [a, b); an explicit Euler step of length dt keeps every new
// value a convex combination of the old ones while dt times it is <= 1.
double diffusion_row_sum_max(long ld, long a, long b, const double* pos, double V, double D,
                             double h) {
  double smax = 0.0;
  for (long i = a; i < b; ++i) {
    double S = 0.0;
    for (long j = a; j < b; ++j) {
      if (j == i) continue;
      const double dx = pos[i] - pos[j], dy = pos[ld + i] - pos[ld + j];
      const double dz = pos[2 * ld + i] - pos[2 * ld + j];
      const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
      if (r >= 2.0 * h) continue;
      S -= 2.0 * D * V * r * wendland_dwdr(r, h) / (r * r + 0.01 * h * h);
    }
    smax = std::max(smax, S);
  }
  return smax;
}

// Substeps for an interval of dt_s seconds: the fewest that keep every update
// a convex combination of the old values, ceil(dt_s S_max), at least 1.
int diffusion_substeps(double dt_s, double smax) {
  const double want = std::ceil(dt_s * smax);
  return want >= 1.0 ? (int)want : 1;
}

// Largest row sum of the operator over all particles of one array (see
// diffusion_row_sum_max).
double oracle_diffusion_row_sum_max(long n, const double* pos, double V, double D, double h) {
  return diffusion_row_sum_max(n, 0, n, pos, V, D, h);
}

// All particles of one array (see diffuse_range).
void oracle_diffuse(long n, const double* pos, double* y, double V, double D, double h,
                    double dt_s, int n_sub) {
  diffuse_range(n, 0, n, pos, y, V, D, h, dt_s, n_sub);
}

// Brute-force reference: classical explicit RK4 with n_steps equal steps.
int oracle_rk4(const double* params, double T, double V_liq, double V_gas, double D,
               const double* y_in, double* y, double dt_days, long n_steps) {
  Model m;
  make_model(params, T, V_liq, V_gas, m);
  Particle P{&m, y_in, D, 1e-7};
  const double h = dt_days / (double)n_steps;
  double k1[NS], k2[NS], k3[NS], k4[NS], tmp[NS];
  for (long s = 0; s < n_steps; ++s) {
    rhs(P, y, k1);
    for (int i = 0; i < NS; ++i) tmp[i] = y[i] + 0.5 * h * k1[i];
    rhs(P, tmp, k2);
    for (int i = 0; i < NS; ++i) tmp[i] = y[i] + 0.5 * h * k2[i];
    rhs(P, tmp, k3);
    for (int i = 0; i < NS; ++i) tmp[i] = y[i] + h * k3[i];
    rhs(P, tmp, k4);
    for (int i = 0; i < NS; ++i) y[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  }
  return P.newton_failed ? ST_NEWTON : 0;
}

void oracle_philox4x64_10(const uint64_t* ctr4, const uint64_t* key2, uint64_t* out4) {
  philox4x64_10(ctr4, key2, out4);
}

double oracle_gauss(uint64_t seed, uint64_t pid, uint64_t interval, uint64_t sub, uint64_t axis) {
  return gauss_irwin_hall(seed, pid, interval, sub, axis);
}

// Population run.  Layouts: y (NS x N SoA), pos (3 x N SoA), params (n_dig x NPARAM),
// flow (n_dig x (7 + NS)): has_flow, U, R, H, sigma, slab_zmin, q_in, y_in[NS].
// D_uniform (n_dig): dilution rate for digesters without flow.
// stats4: accepted, rejected, newton iterations, bisections (summed).
int oracle_run(int n_dig, const long* dig_offset, const double* params, const double* V_liq,
               const double* V_gas, const double* D_uniform, const double* flow,
               const uint64_t* flow_seed, int shared_headspace, long N, double* pos,
               double* y, const double* T, double* SH, double* h, int* status,
               double dt_coupling_s, int n_intervals, long interval0, double rtol,
               const double* atol, long max_steps, int fixed_n, int n_threads,
               long* stats4, int h2_alg, const double* diff_D, const double* diff_h) {
  if (n_threads <= 0) n_threads = (int)std::max(1u, std::thread::hardware_concurrency());
  const int FL = 7 + NS;
  const double dt_days = dt_coupling_s / 86400.0;
  std::vector<int> dig_of(N);
  for (int d = 0; d < n_dig; ++d)
    for (long p = dig_offset[d]; p < dig_offset[d + 1]; ++p) dig_of[p] = d;
  // per-digester advection constants (computed once per run, as in the library)
  std::vector<Flow> fl(n_dig);
  std::vector<double> cs(n_dig), sn(n_dig), D_slab(n_dig);
  int n_sub = (int)std::lround(dt_coupling_s);
  if (n_sub < 1) n_sub = 1;
  const double dsub = dt_coupling_s / n_sub;
  for (int d = 0; d < n_dig; ++d) {
    const double* r = flow + (long)d * FL;
    fl[d] = Flow{r[0] != 0.0, r[1], r[2], r[3], r[4], r[5], r[6], r + 7, flow_seed[d]};
    double w = fl[d].on ? fl[d].U / fl[d].R : 0.0;
    cs[d] = std::cos(w * dsub);
    sn[d] = std::sin(w * dsub);
    D_slab[d] = fl[d].on ? fl[d].q_in / (M_PI * fl[d].R * fl[d].R * (fl[d].H - fl[d].slab_zmin)) : 0.0;
  }
  std::vector<long> acc(N, 0), rej(N, 0), nit(N, 0), nbis(N, 0);
  std::vector<double> Dp(N);
  bool any_diff = false;
  if (diff_D)
    for (int d = 0; d < n_dig; ++d)
      any_diff |= diff_D[d] > 0.0 && dig_offset[d + 1] > dig_offset[d];
  for (int it = 0; it < n_intervals; ++it) {
    const uint64_t gint = (uint64_t)(interval0 + it);
    // advection (positions and the interval's dilution rate)
    parallel_chunks(N, n_threads, [&](long a, long b) {
      for (long p = a; p < b; ++p) {
        const int d = dig_of[p];
        double D = D_uniform[d];
        double* px = pos + p;
        double* py = pos + N + p;
        double* pz = pos + 2 * N + p;
        if (fl[d].on) {
          D = (*pz >= fl[d].slab_zmin) ? D_slab[d] : 0.0;
          advect_one(fl[d], cs[d], sn[d], n_sub, dsub, (uint64_t)(p - dig_offset[d]), gint,
                     *px, *py, *pz);
        }
        Dp[p] = D;
      }
    });
    // diffusion between the particles of each digester; one substep count
    // for all digesters, from the largest row sum over all of them at the
    // interval's positions
    if (any_diff) {
      double smax = 0.0;
      for (int d = 0; d < n_dig; ++d) {
        const long a = dig_offset[d], b = dig_offset[d + 1];
        if (!(diff_D[d] > 0.0) || b <= a) continue;
        smax = std::max(smax, diffusion_row_sum_max(N, a, b, pos, V_liq[d] / (double)(b - a),
                                                    diff_D[d], diff_h[d]));
      }
      const int diff_sub = diffusion_substeps(dt_coupling_s, smax);
      for (int d = 0; d < n_dig; ++d) {
        const long a = dig_offset[d], b = dig_offset[d + 1];
        if (!(diff_D[d] > 0.0) || b <= a) continue;
        diffuse_range(N, a, b, pos, y, V_liq[d] / (double)(b - a), diff_D[d], diff_h[d],
                      dt_coupling_s, diff_sub);
      }
    }
    // ADM1 on every particle
    parallel_chunks(N, n_threads, [&](long a, long b) {
      for (long p = a; p < b; ++p) {
        const int d = dig_of[p];
        const double* prm = params + (long)d * NPARAM;
        const double D = Dp[p];
        const double* yin = fl[d].y_in;
        Model m;
        make_model(prm, T[p], V_liq[d], V_gas[d], m);
        double yy[NS];
        for (int i = 0; i < NS; ++i) yy[i] = y[(long)i * N + p];
        Particle P{&m, yin, D, SH[p]};
        P.h2_alg = h2_alg != 0;
        P.SH2 = yy[S_h2];
        StepStats st;
        double hp = h[p];
        int s = integrate_interval(P, yy, &hp, dt_days, rtol, atol, max_steps, fixed_n, st);
        for (int i = 0; i < NS; ++i) y[(long)i * N + p] = yy[i];
        h[p] = hp;
        SH[p] = P.SH;
        status[p] |= s;
        acc[p] += st.accepted; rej[p] += st.rejected;
        nit[p] += P.ns.iters; nbis[p] += P.ns.bisections;
      }
    });
    if (shared_headspace) {
      // volume-weighted (equal volumes within a digester) mean of the gas
      // states, compensated summation, written back to every particle
      for (int d = 0; d < n_dig; ++d) {
        long a = dig_offset[d], b = dig_offset[d + 1];
        if (b <= a) continue;
        for (int g = G_h2; g <= G_co2; ++g) {
          double s = 0.0, c = 0.0;
          for (long p = a; p < b; ++p) {
            double v = y[(long)g * N + p];
            double t = s + v;
            if (std::fabs(s) >= std::fabs(v)) c += (s - t) + v; else c += (v - t) + s;
            s = t;
          }
          double mean = (s + c) / (double)(b - a);
          for (long p = a; p < b; ++p) y[(long)g * N + p] = mean;
        }
      }
    }
  }
  int any = 0;
  long s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (long p = 0; p < N; ++p) {
    any |= status[p];
    s0 += acc[p]; s1 += rej[p]; s2 += nit[p]; s3 += nbis[p];
  }
  if (stats4) { stats4[0] = s0; stats4[1] = s1; stats4[2] = s2; stats4[3] = s3; }
  return any;
}

}  // extern "C"
