// Per-digester ADM1 constants of the CUDA library and their derivation from
// the raw parameter vector (host side).  Sec. 2.2 of the paper: Eq. 2 mass
// balances with the standard ADM1 stoichiometry, Eq. 3-6 inhibitions, Eq. 7
// charge balance.  Temperature-dependent constants are completed per
// particle on the device (see adm1_device.cuh).
#pragma once
#include <cstdint>

namespace chad {

constexpr int NS = 29;
constexpr int kPartConstFields = 9;  // PartConst fields stored per particle

// state indices (Sec. 2.2; 12 solubles, 12 particulates, 2 ions, 3 gases)
enum : int {
  iS_su, iS_aa, iS_fa, iS_va, iS_bu, iS_pro, iS_ac, iS_h2, iS_ch4, iS_IC, iS_IN, iS_I,
  iX_c, iX_ch, iX_pr, iX_li, iX_su, iX_aa, iX_fa, iX_c4, iX_pro, iX_ac, iX_h2, iX_I,
  iS_cat, iS_an, iG_h2, iG_ch4, iG_co2
};

// Raw parameter layout of one digester (names exported by chad_param_name).
#define CHAD_PARAM_LIST(X)                                                          \
  X(f_sI_xc) X(f_xI_xc) X(f_ch_xc) X(f_pr_xc) X(f_li_xc)                            \
  X(N_xc) X(N_I) X(N_aa) X(N_bac)                                                   \
  X(C_xc) X(C_sI) X(C_ch) X(C_pr) X(C_li) X(C_xI) X(C_su) X(C_aa) X(C_fa)           \
  X(C_bu) X(C_pro) X(C_ac) X(C_bac) X(C_va) X(C_ch4)                                \
  X(f_fa_li) X(f_h2_su) X(f_bu_su) X(f_pro_su) X(f_ac_su)                           \
  X(f_h2_aa) X(f_va_aa) X(f_bu_aa) X(f_pro_aa) X(f_ac_aa)                           \
  X(f_ac_fa) X(f_h2_fa) X(f_pro_va) X(f_ac_va) X(f_h2_va) X(f_ac_bu) X(f_h2_bu)     \
  X(f_ac_pro) X(f_h2_pro)                                                           \
  X(Y_su) X(Y_aa) X(Y_fa) X(Y_c4) X(Y_pro) X(Y_ac) X(Y_h2)                          \
  X(k_dis) X(k_hyd_ch) X(k_hyd_pr) X(k_hyd_li)                                      \
  X(k_m_su) X(k_m_aa) X(k_m_fa) X(k_m_c4) X(k_m_pro) X(k_m_ac) X(k_m_h2)            \
  X(k_dec_X_su) X(k_dec_X_aa) X(k_dec_X_fa) X(k_dec_X_c4) X(k_dec_X_pro)            \
  X(k_dec_X_ac) X(k_dec_X_h2)                                                       \
  X(K_S_IN) X(K_S_su) X(K_S_aa) X(K_S_fa) X(K_S_c4) X(K_S_pro) X(K_S_ac) X(K_S_h2)  \
  X(K_I_h2_fa) X(K_I_h2_c4) X(K_I_h2_pro) X(K_I_nh3)                                \
  X(pH_LL_aa) X(pH_UL_aa) X(pH_LL_ac) X(pH_UL_ac) X(pH_LL_h2) X(pH_UL_h2)           \
  X(R) X(R_J) X(T_base)                                                             \
  X(pK_w) X(pK_a_va) X(pK_a_bu) X(pK_a_pro) X(pK_a_ac) X(pK_a_co2) X(pK_a_IN)       \
  X(dH_K_w) X(dH_K_a_co2) X(dH_K_a_IN)                                              \
  X(K_H_co2) X(K_H_ch4) X(K_H_h2) X(dH_K_H_co2) X(dH_K_H_ch4) X(dH_K_H_h2)          \
  X(p_h2o_base) X(p_h2o_theta)                                                      \
  X(k_La) X(k_p) X(V_liq_ref) X(P_atm)                                              \
  X(Ea_over_R) X(T_ref_kin)

enum ParamIndex : int {
#define CHAD_X(n) p_##n,
  CHAD_PARAM_LIST(CHAD_X)
#undef CHAD_X
  kNumParams
};

// Temperature-independent constants of one digester, laid out for the device.
// T = T is the model's precision; the mixed form keeps a float copy for
// its FP32 Jacobian evaluation (each FP64->FP32 conversion there would take an
// FP64 pipe slot).  All members are T except the four ints.
template <class T>
struct DigConstT {
  // kinetics at the reference temperature (1/d) and their Arrhenius scaling
  T k_dis, k_hyd_ch, k_hyd_pr, k_hyd_li;
  T k_m_su, k_m_aa, k_m_fa, k_m_c4, k_m_pro, k_m_ac, k_m_h2;
  T k_dec[7];
  T Ea_over_R, inv_T_ref;
  T K_S_IN, K_S_su, K_S_aa, K_S_fa, K_S_c4, K_S_pro, K_S_ac, K_S_h2;
  T K_I_h2_fa, K_I_h2_c4, K_I_h2_pro, K_I_nh3;
  // Hill pH inhibition I = 1 / (1 + (S_H / K_pH)^n)
  T inv_K_pH_aa, inv_K_pH_ac, inv_K_pH_h2;
  T n_aa, n_ac, n_h2;
  int ni_aa, ni_ac, ni_h2;  // n as a small integer (1..4), or 0 if not integral
  int pad0;
  // acid-base and gas-liquid constants
  T K_a_va, K_a_bu, K_a_pro, K_a_ac;                       // T-independent
  T K_w_b, K_a_co2_b, K_a_IN_b, K_H_co2_b, K_H_ch4_b, K_H_h2_b, p_h2o_b;  // at T_base
  T th_w, th_a_co2, th_a_IN, th_H_co2, th_H_ch4, th_H_h2, th_h2o;        // dH/R (K)
  T inv_T_base, R, P_atm, k_La, kp_over_Vgas, Vliq_over_Vgas;
  // stoichiometric coefficients of the mass balances
  T f_sI, f_xI, f_ch, f_pr, f_li, c_su_li, f_fa_li;
  T su_h2, su_bu, su_pro, su_ac, Y_su;   // (1 - Y_su) f_x,su
  T aa_h2, aa_va, aa_bu, aa_pro, aa_ac, Y_aa;
  T fa_h2, fa_ac, Y_fa;
  T va_pro, va_ac, va_h2, bu_ac, bu_h2, Y_c4;
  T pro_ac, pro_h2, Y_pro;
  T ac_ch4, Y_ac, h2_ch4, Y_h2;
  T cIC[13];  // S_IC coefficient of processes 1..12 and decay (13)
  T nIN[13];  // S_IN coefficient of processes 1..12 and decay (13)
  // inflow
  T y_in[NS];
  T D_uniform;
};
using DigConst = DigConstT<double>;
using DigConstF = DigConstT<float>;

// Float copy of a digester's constants (rounded to nearest).
void narrow_digester(const DigConst& d, DigConstF& f);

// Flow field of one digester, expanded for the device.
struct FlowConst {
  int has_flow, n_sub;
  double U, sigma;   // swirl speed at r = R (m/s) and noise std (m/s)
  double cw, sw;     // cos / sin of the rotation per sub-step
  double amp;        // sigma * sub-step length (m)
  double R, H, slab_zmin, D_slab;
  uint64_t seed;
};

// Fill a DigConst from raw parameters.  Returns false for invalid values.
bool derive_digester(const double* p, double V_liq, double V_gas, double D_uniform,
                     const double* y_in, DigConst& c, const char** why);

extern const char* const kParamNames[kNumParams];

}  // namespace chad
