// Host-side derivation of the per-digester ADM1 constants (Sec. 2.2).
// Stoichiometric coefficients follow the standard ADM1 mass balances that
// the paper takes from its Ref. [14]; the S_IC and S_IN coefficients are the
// carbon and nitrogen balances of each process written out term by term.
#include <cmath>
#include <cstddef>
#include <cstring>

#include "model.h"

namespace chad {

const char* const kParamNames[kNumParams] = {
#define CHAD_X(n) #n,
    CHAD_PARAM_LIST(CHAD_X)
#undef CHAD_X
};

static int small_integer(double n) {
  for (int k = 1; k <= 4; ++k)
    if (n == (double)k) return k;
  return 0;
}

bool derive_digester(const double* p, double V_liq, double V_gas, double D_uniform,
                     const double* y_in, DigConst& c, const char** why) {
  std::memset(&c, 0, sizeof(c));
  for (int i = 0; i < kNumParams; ++i) {
    if (!std::isfinite(p[i])) {
      *why = "non-finite parameter";
      return false;
    }
  }
  if (!(V_liq > 0.0) || !(V_gas > 0.0)) { *why = "V_liq and V_gas must be > 0"; return false; }
  if (!(D_uniform >= 0.0) || !std::isfinite(D_uniform)) { *why = "D_uniform must be >= 0"; return false; }
  if (!(p[p_T_base] > 0.0) || !(p[p_T_ref_kin] > 0.0) || !(p[p_R_J] > 0.0) || !(p[p_P_atm] > 0.0)) {
    *why = "T_base, T_ref_kin, R_J and P_atm must be > 0";
    return false;
  }
  const double pos_list[] = {p[p_K_S_IN], p[p_K_S_su], p[p_K_S_aa], p[p_K_S_fa], p[p_K_S_c4],
                             p[p_K_S_pro], p[p_K_S_ac], p[p_K_S_h2], p[p_K_I_h2_fa],
                             p[p_K_I_h2_c4], p[p_K_I_h2_pro], p[p_K_I_nh3]};
  for (double v : pos_list)
    if (!(v > 0.0)) { *why = "half-saturation and inhibition constants must be > 0"; return false; }
  if (!(p[p_pH_UL_aa] > p[p_pH_LL_aa]) || !(p[p_pH_UL_ac] > p[p_pH_LL_ac]) ||
      !(p[p_pH_UL_h2] > p[p_pH_LL_h2])) {
    *why = "pH upper limits must exceed lower limits";
    return false;
  }

  c.k_dis = p[p_k_dis];
  c.k_hyd_ch = p[p_k_hyd_ch];
  c.k_hyd_pr = p[p_k_hyd_pr];
  c.k_hyd_li = p[p_k_hyd_li];
  c.k_m_su = p[p_k_m_su];
  c.k_m_aa = p[p_k_m_aa];
  c.k_m_fa = p[p_k_m_fa];
  c.k_m_c4 = p[p_k_m_c4];
  c.k_m_pro = p[p_k_m_pro];
  c.k_m_ac = p[p_k_m_ac];
  c.k_m_h2 = p[p_k_m_h2];
  c.k_dec[0] = p[p_k_dec_X_su];
  c.k_dec[1] = p[p_k_dec_X_aa];
  c.k_dec[2] = p[p_k_dec_X_fa];
  c.k_dec[3] = p[p_k_dec_X_c4];
  c.k_dec[4] = p[p_k_dec_X_pro];
  c.k_dec[5] = p[p_k_dec_X_ac];
  c.k_dec[6] = p[p_k_dec_X_h2];
  c.Ea_over_R = p[p_Ea_over_R];
  c.inv_T_ref = 1.0 / p[p_T_ref_kin];
  c.K_S_IN = p[p_K_S_IN];
  c.K_S_su = p[p_K_S_su];
  c.K_S_aa = p[p_K_S_aa];
  c.K_S_fa = p[p_K_S_fa];
  c.K_S_c4 = p[p_K_S_c4];
  c.K_S_pro = p[p_K_S_pro];
  c.K_S_ac = p[p_K_S_ac];
  c.K_S_h2 = p[p_K_S_h2];
  c.K_I_h2_fa = p[p_K_I_h2_fa];
  c.K_I_h2_c4 = p[p_K_I_h2_c4];
  c.K_I_h2_pro = p[p_K_I_h2_pro];
  c.K_I_nh3 = p[p_K_I_nh3];

  // Hill form in concentration units: K_pH = 10^-(LL+UL)/2, n = 3/(UL-LL)
  c.inv_K_pH_aa = std::pow(10.0, 0.5 * (p[p_pH_LL_aa] + p[p_pH_UL_aa]));
  c.inv_K_pH_ac = std::pow(10.0, 0.5 * (p[p_pH_LL_ac] + p[p_pH_UL_ac]));
  c.inv_K_pH_h2 = std::pow(10.0, 0.5 * (p[p_pH_LL_h2] + p[p_pH_UL_h2]));
  c.n_aa = 3.0 / (p[p_pH_UL_aa] - p[p_pH_LL_aa]);
  c.n_ac = 3.0 / (p[p_pH_UL_ac] - p[p_pH_LL_ac]);
  c.n_h2 = 3.0 / (p[p_pH_UL_h2] - p[p_pH_LL_h2]);
  c.ni_aa = small_integer(c.n_aa);
  c.ni_ac = small_integer(c.n_ac);
  c.ni_h2 = small_integer(c.n_h2);

  c.K_a_va = std::pow(10.0, -p[p_pK_a_va]);
  c.K_a_bu = std::pow(10.0, -p[p_pK_a_bu]);
  c.K_a_pro = std::pow(10.0, -p[p_pK_a_pro]);
  c.K_a_ac = std::pow(10.0, -p[p_pK_a_ac]);
  c.K_w_b = std::pow(10.0, -p[p_pK_w]);
  c.K_a_co2_b = std::pow(10.0, -p[p_pK_a_co2]);
  c.K_a_IN_b = std::pow(10.0, -p[p_pK_a_IN]);
  c.K_H_co2_b = p[p_K_H_co2];
  c.K_H_ch4_b = p[p_K_H_ch4];
  c.K_H_h2_b = p[p_K_H_h2];
  c.p_h2o_b = p[p_p_h2o_base];
  const double RJ = p[p_R_J];
  c.th_w = p[p_dH_K_w] / RJ;
  c.th_a_co2 = p[p_dH_K_a_co2] / RJ;
  c.th_a_IN = p[p_dH_K_a_IN] / RJ;
  c.th_H_co2 = p[p_dH_K_H_co2] / RJ;
  c.th_H_ch4 = p[p_dH_K_H_ch4] / RJ;
  c.th_H_h2 = p[p_dH_K_H_h2] / RJ;
  c.th_h2o = p[p_p_h2o_theta];
  c.inv_T_base = 1.0 / p[p_T_base];
  c.R = p[p_R];
  c.P_atm = p[p_P_atm];
  c.k_La = p[p_k_La];
  // k_p is given for a tank of V_liq_ref; it scales with the liquid volume,
  // and every particle carries the same share of liquid and gas (Sec. 2.3)
  c.kp_over_Vgas = p[p_k_p] * (V_liq / p[p_V_liq_ref]) / V_gas;
  c.Vliq_over_Vgas = V_liq / V_gas;

  // stoichiometry
  const double Ysu = p[p_Y_su], Yaa = p[p_Y_aa], Yfa = p[p_Y_fa], Yc4 = p[p_Y_c4];
  const double Ypro = p[p_Y_pro], Yac = p[p_Y_ac], Yh2 = p[p_Y_h2];
  c.f_sI = p[p_f_sI_xc];
  c.f_xI = p[p_f_xI_xc];
  c.f_ch = p[p_f_ch_xc];
  c.f_pr = p[p_f_pr_xc];
  c.f_li = p[p_f_li_xc];
  c.f_fa_li = p[p_f_fa_li];
  c.c_su_li = 1.0 - p[p_f_fa_li];
  c.su_h2 = (1.0 - Ysu) * p[p_f_h2_su];
  c.su_bu = (1.0 - Ysu) * p[p_f_bu_su];
  c.su_pro = (1.0 - Ysu) * p[p_f_pro_su];
  c.su_ac = (1.0 - Ysu) * p[p_f_ac_su];
  c.Y_su = Ysu;
  c.aa_h2 = (1.0 - Yaa) * p[p_f_h2_aa];
  c.aa_va = (1.0 - Yaa) * p[p_f_va_aa];
  c.aa_bu = (1.0 - Yaa) * p[p_f_bu_aa];
  c.aa_pro = (1.0 - Yaa) * p[p_f_pro_aa];
  c.aa_ac = (1.0 - Yaa) * p[p_f_ac_aa];
  c.Y_aa = Yaa;
  c.fa_h2 = (1.0 - Yfa) * p[p_f_h2_fa];
  c.fa_ac = (1.0 - Yfa) * p[p_f_ac_fa];
  c.Y_fa = Yfa;
  c.va_pro = (1.0 - Yc4) * p[p_f_pro_va];
  c.va_ac = (1.0 - Yc4) * p[p_f_ac_va];
  c.va_h2 = (1.0 - Yc4) * p[p_f_h2_va];
  c.bu_ac = (1.0 - Yc4) * p[p_f_ac_bu];
  c.bu_h2 = (1.0 - Yc4) * p[p_f_h2_bu];
  c.Y_c4 = Yc4;
  c.pro_ac = (1.0 - Ypro) * p[p_f_ac_pro];
  c.pro_h2 = (1.0 - Ypro) * p[p_f_h2_pro];
  c.Y_pro = Ypro;
  c.ac_ch4 = 1.0 - Yac;
  c.Y_ac = Yac;
  c.h2_ch4 = 1.0 - Yh2;
  c.Y_h2 = Yh2;

  // Carbon: the inorganic carbon released by process j is minus the carbon
  // of its organic products and substrates (kmol C per kgCOD contents).
  const double Cxc = p[p_C_xc], CsI = p[p_C_sI], Cch = p[p_C_ch], Cpr = p[p_C_pr];
  const double Cli = p[p_C_li], CxI = p[p_C_xI], Csu = p[p_C_su], Caa = p[p_C_aa];
  const double Cfa = p[p_C_fa], Cbu = p[p_C_bu], Cpro = p[p_C_pro], Cac = p[p_C_ac];
  const double Cbac = p[p_C_bac], Cva = p[p_C_va], Cch4 = p[p_C_ch4];
  double s[13];
  s[0] = -Cxc + c.f_sI * CsI + c.f_ch * Cch + c.f_pr * Cpr + c.f_li * Cli + c.f_xI * CxI;
  s[1] = -Cch + Csu;
  s[2] = -Cpr + Caa;
  s[3] = -Cli + c.c_su_li * Csu + c.f_fa_li * Cfa;
  s[4] = -Csu + c.su_bu * Cbu + c.su_pro * Cpro + c.su_ac * Cac + Ysu * Cbac;
  s[5] = -Caa + c.aa_va * Cva + c.aa_bu * Cbu + c.aa_pro * Cpro + c.aa_ac * Cac + Yaa * Cbac;
  s[6] = -Cfa + c.fa_ac * Cac + Yfa * Cbac;
  s[7] = -Cva + c.va_pro * Cpro + c.va_ac * Cac + Yc4 * Cbac;
  s[8] = -Cbu + c.bu_ac * Cac + Yc4 * Cbac;
  s[9] = -Cpro + c.pro_ac * Cac + Ypro * Cbac;
  s[10] = -Cac + c.ac_ch4 * Cch4 + Yac * Cbac;
  s[11] = c.h2_ch4 * Cch4 + Yh2 * Cbac;
  s[12] = -Cbac + Cxc;
  for (int j = 0; j < 13; ++j) c.cIC[j] = -s[j];

  // Nitrogen: N_xc, N_I, N_aa, N_bac are contents per kgCOD
  const double Nxc = p[p_N_xc], NI = p[p_N_I], Naa = p[p_N_aa], Nbac = p[p_N_bac];
  c.nIN[0] = Nxc - c.f_xI * NI - c.f_sI * NI - c.f_pr * Naa;
  c.nIN[1] = 0.0;
  c.nIN[2] = 0.0;
  c.nIN[3] = 0.0;
  c.nIN[4] = -Ysu * Nbac;
  c.nIN[5] = Naa - Yaa * Nbac;
  c.nIN[6] = -Yfa * Nbac;
  c.nIN[7] = -Yc4 * Nbac;
  c.nIN[8] = -Yc4 * Nbac;
  c.nIN[9] = -Ypro * Nbac;
  c.nIN[10] = -Yac * Nbac;
  c.nIN[11] = -Yh2 * Nbac;
  c.nIN[12] = Nbac - Nxc;

  for (int i = 0; i < NS; ++i) {
    const double v = y_in ? y_in[i] : 0.0;
    if (!std::isfinite(v)) { *why = "non-finite influent"; return false; }
    c.y_in[i] = v;
  }
  c.D_uniform = D_uniform;
  return true;
}

// The members are all of the element type except the block of four ints
// (ni_aa .. pad0), which K_a_va follows; the copy walks the two runs.
void narrow_digester(const DigConst& d, DigConstF& f) {
  constexpr size_t nb = offsetof(DigConst, ni_aa) / sizeof(double);
  constexpr size_t na = (sizeof(DigConst) - offsetof(DigConst, K_a_va)) / sizeof(double);
  static_assert(offsetof(DigConstF, ni_aa) == nb * sizeof(float), "DigConstT layout");
  static_assert((sizeof(DigConstF) - offsetof(DigConstF, K_a_va)) / sizeof(float) == na,
                "DigConstT layout");
  static_assert(offsetof(DigConst, K_a_va) - offsetof(DigConst, ni_aa) == 4 * sizeof(int),
                "DigConstT layout");
  const double* db = reinterpret_cast<const double*>(&d);
  float* fb = reinterpret_cast<float*>(&f);
  for (size_t i = 0; i < nb; ++i) fb[i] = (float)db[i];
  f.ni_aa = d.ni_aa;
  f.ni_ac = d.ni_ac;
  f.ni_h2 = d.ni_h2;
  f.pad0 = d.pad0;
  const double* da = reinterpret_cast<const double*>(reinterpret_cast<const char*>(&d) +
                                                     offsetof(DigConst, K_a_va));
  float* fa = reinterpret_cast<float*>(reinterpret_cast<char*>(&f) + offsetof(DigConstF, K_a_va));
  for (size_t i = 0; i < na; ++i) fa[i] = (float)da[i];
}

}  // namespace chad
