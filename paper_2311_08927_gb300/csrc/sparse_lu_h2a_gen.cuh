// GENERATED by gen_sparse.py from the library's own Jacobian pattern -- do not edit.
// Static-order (Markowitz) sparse LU of W_d = I - g J_d without the S_h2 row and
// column (S_h2 algebraic, Eq. 8: those go to a second Sherman-Morrison level),
// over the other 28 ADM1 states (J_d: the Jacobian with S_H held fixed).
// pattern nnz(J_d) = 146, slots with fill = 167
#pragma once
#include "adm1_device.cuh"

namespace chad {
namespace spa {

constexpr int kNNZ = 167;
constexpr int kNNZ_J = 146;
constexpr int kPiv = 28;  // pivots (every state but S_h2)
// slots of the Jacobian scatter: the LU's, then the S_h2 row (kNNZ + c)
// and the S_h2 column (kNNZ + NS + r)
constexpr int kStore = 225;
// elimination position -> state index
constexpr int kOrder[kPiv] = {11, 23, 24, 25, 13, 14, 15, 22, 8, 26, 27, 28, 9, 21, 18, 2, 20, 16, 0, 17, 1, 6, 5, 12, 3, 4, 10, 19};

CHAD_HD constexpr int slot(int r, int c) {
  // row-major table over states, -1 = structurally zero
  const int t[NS * NS] = {
      78, -1, -1, -1, -1, -1, -1, 196, -1, -1, 80, -1, 79, 75, -1, 76, 77, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, 86, -1, -1, -1, -1, -1, 197, -1, -1, 88, -1, 87, -1, 84, -1, -1, 85, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, 66, -1, -1, -1, -1, 198, -1, -1, 68, -1, 67, -1, -1, 64, -1, -1, 65, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, 132, -1, 134, 135, -1, -1, 199, -1, -1, 136, -1, 133, -1, -1, -1, -1, 131, -1, 137, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      139, 141, -1, 143, 144, -1, -1, 200, -1, -1, 145, -1, 142, -1, -1, -1, 138, 140, -1, 146, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      106, 108, -1, 111, 112, 109, -1, 201, -1, -1, 113, -1, 110, -1, -1, -1, 105, 107, -1, 114, 104, -1, -1, -1, -1, -1, -1, -1, -1,
      94, 96, 91, 100, 101, 98, 97, 202, -1, -1, 102, -1, 99, -1, -1, -1, 93, 95, 90, 103, 92, 89, -1, -1, -1, -1, -1, -1, -1,
      167, 168, 169, 170, 171, 172, 173, 174, 175, 176, 177, 178, 179, 180, 181, 182, 183, 184, 185, 186, 187, 188, 189, 190, 191, 192, 193, 194, 195,
      -1, -1, -1, -1, -1, -1, 18, 204, 15, -1, 19, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 17, 14, -1, -1, -1, -1, 16, -1,
      48, 50, 45, 54, 55, 52, 51, 205, -1, 42, 56, -1, 53, 37, 38, 39, 47, 49, 44, 57, 46, 43, 40, -1, -1, -1, -1, -1, 41,
      153, 155, 150, 159, 160, 157, 156, 206, -1, -1, 161, -1, 158, -1, -1, -1, 152, 154, 149, 162, 151, 148, 147, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, 207, -1, -1, -1, 0, 1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      121, 123, 118, 127, 128, 125, 124, 208, -1, -1, 129, -1, 126, -1, -1, -1, 120, 122, 117, 130, 119, 116, 115, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, 209, -1, -1, -1, -1, 7, 6, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, 210, -1, -1, -1, -1, 9, -1, 8, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, 211, -1, -1, -1, -1, 11, -1, -1, 10, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      73, -1, -1, -1, -1, -1, -1, 212, -1, -1, 74, -1, -1, -1, -1, -1, 72, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, 82, -1, -1, -1, -1, -1, 213, -1, -1, 83, -1, -1, -1, -1, -1, -1, 81, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, 62, -1, -1, -1, -1, 214, -1, -1, 63, -1, -1, -1, -1, -1, -1, -1, 61, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, 163, 164, -1, -1, 215, -1, -1, 165, -1, -1, -1, -1, -1, -1, -1, -1, 166, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, 70, -1, 216, -1, -1, 71, -1, -1, -1, -1, -1, -1, -1, -1, -1, 69, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, 59, 217, -1, -1, 60, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 58, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, 218, -1, -1, 13, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 12, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, 219, -1, -1, -1, -1, 3, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 2, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, 220, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 4, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, 221, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 5, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, 222, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 20, 21, 22,
      -1, -1, -1, -1, -1, -1, 28, 223, 23, -1, 29, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 27, -1, -1, -1, -1, 24, 25, 26,
      -1, -1, -1, -1, -1, -1, 35, 224, -1, 33, 36, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 34, -1, -1, -1, -1, 30, 31, 32
  };
  return t[r * NS + c];
}

struct Idx {
  static CHAD_HD constexpr int at(int r, int c) { return slot(r, c); }
  static constexpr int size = kStore;
};

// diagonal slots in elimination order
constexpr int kDiag[kPiv] = {0, 2, 4, 5, 6, 8, 10, 12, 15, 20, 25, 32, 42, 58, 61, 66, 69, 72, 78, 81, 86, 97, 109, 126, 134, 144, 161, 166};

// W_d = I - g J_d in place over the slots (fill slots hold zero in J_d).
// W: the slot storage, a pointer or any accessor whose w[s] is a reference.
template <class R, class W>
CHAD_HD void form_w(W w, R g) {
#pragma unroll
  for (int s = 0; s < kNNZ; ++s) w[s] = -g * w[s];
  w[0] += R(1);
  w[2] += R(1);
  w[4] += R(1);
  w[5] += R(1);
  w[6] += R(1);
  w[8] += R(1);
  w[10] += R(1);
  w[12] += R(1);
  w[15] += R(1);
  w[20] += R(1);
  w[25] += R(1);
  w[32] += R(1);
  w[42] += R(1);
  w[58] += R(1);
  w[61] += R(1);
  w[66] += R(1);
  w[69] += R(1);
  w[72] += R(1);
  w[78] += R(1);
  w[81] += R(1);
  w[86] += R(1);
  w[97] += R(1);
  w[109] += R(1);
  w[126] += R(1);
  w[134] += R(1);
  w[144] += R(1);
  w[161] += R(1);
  w[166] += R(1);
}

// In-place LU; the diagonal slots receive the reciprocals of the pivots
// (the only use the solve makes of them).  Returns false if a pivot fails
// the threshold test.
template <class R, class W>
CHAD_HD bool factor(W w) {
  using P = PivTest<R>;
  bool ok = true;
  {  // pivot 0: state 11 (S_I), 0 rows x 1 cols
    const R pv = w[0];
    ok = ok && P::good(P::key(pv));
    const R inv = rcp<R>(pv);
    w[0] = inv;
  }
  {  // pivot 1: state 23 (X_I), 0 rows x 1 cols
    const R pv = w[2];
    ok = ok && P::good(P::key(pv));
    const R inv = rcp<R>(pv);
    w[2] = inv;
  }
  {  // pivot 2: state 24 (S_cat), 0 rows x 0 cols
    const R pv = w[4];
    ok = ok && P::good(P::key(pv));
    const R inv = rcp<R>(pv);
    w[4] = inv;
  }
  {  // pivot 3: state 25 (S_an), 0 rows x 0 cols
    const R pv = w[5];
    ok = ok && P::good(P::key(pv));
    const R inv = rcp<R>(pv);
    w[5] = inv;
  }
  {  // pivot 4: state 13 (X_ch), 2 rows x 1 cols
    const R pv = w[6];
    const typename P::K cm = P::kmax(P::key(w[37]), P::key(w[75]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[6] = inv;
    { const R l = w[37] * inv; w[37] = l;
      w[53] -= l * w[7];
    }
    { const R l = w[75] * inv; w[75] = l;
      w[79] -= l * w[7];
    }
  }
  {  // pivot 5: state 14 (X_pr), 2 rows x 1 cols
    const R pv = w[8];
    const typename P::K cm = P::kmax(P::key(w[38]), P::key(w[84]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[8] = inv;
    { const R l = w[38] * inv; w[38] = l;
      w[53] -= l * w[9];
    }
    { const R l = w[84] * inv; w[84] = l;
      w[87] -= l * w[9];
    }
  }
  {  // pivot 6: state 15 (X_li), 3 rows x 1 cols
    const R pv = w[10];
    const typename P::K cm = P::kmax(P::kmax(P::key(w[39]), P::key(w[64])), P::key(w[76]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[10] = inv;
    { const R l = w[39] * inv; w[39] = l;
      w[53] -= l * w[11];
    }
    { const R l = w[64] * inv; w[64] = l;
      w[67] -= l * w[11];
    }
    { const R l = w[76] * inv; w[76] = l;
      w[79] -= l * w[11];
    }
  }
  {  // pivot 7: state 22 (X_h2), 4 rows x 1 cols
    const R pv = w[12];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::key(w[14]), P::key(w[40])), P::key(w[115])), P::key(w[147]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[12] = inv;
    { const R l = w[14] * inv; w[14] = l;
      w[19] -= l * w[13];
    }
    { const R l = w[40] * inv; w[40] = l;
      w[56] -= l * w[13];
    }
    { const R l = w[115] * inv; w[115] = l;
      w[129] -= l * w[13];
    }
    { const R l = w[147] * inv; w[147] = l;
      w[161] -= l * w[13];
    }
  }
  {  // pivot 8: state 8 (S_ch4), 1 rows x 4 cols
    const R pv = w[15];
    const typename P::K cm = P::key(w[23]);
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[15] = inv;
    { const R l = w[23] * inv; w[23] = l;
      w[25] -= l * w[16];
      w[27] -= l * w[17];
      w[28] -= l * w[18];
      w[29] -= l * w[19];
    }
  }
  {  // pivot 9: state 26 (S_gas_h2), 2 rows x 2 cols
    const R pv = w[20];
    const typename P::K cm = P::kmax(P::key(w[24]), P::key(w[30]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[20] = inv;
    { const R l = w[24] * inv; w[24] = l;
      w[25] -= l * w[21];
      w[26] -= l * w[22];
    }
    { const R l = w[30] * inv; w[30] = l;
      w[31] -= l * w[21];
      w[32] -= l * w[22];
    }
  }
  {  // pivot 10: state 27 (S_gas_ch4), 1 rows x 4 cols
    const R pv = w[25];
    const typename P::K cm = P::key(w[31]);
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[25] = inv;
    { const R l = w[31] * inv; w[31] = l;
      w[32] -= l * w[26];
      w[34] -= l * w[27];
      w[35] -= l * w[28];
      w[36] -= l * w[29];
    }
  }
  {  // pivot 11: state 28 (S_gas_co2), 1 rows x 4 cols
    const R pv = w[32];
    const typename P::K cm = P::key(w[41]);
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[32] = inv;
    { const R l = w[41] * inv; w[41] = l;
      w[42] -= l * w[33];
      w[43] -= l * w[34];
      w[51] -= l * w[35];
      w[56] -= l * w[36];
    }
  }
  {  // pivot 12: state 9 (S_IC), 0 rows x 15 cols
    const R pv = w[42];
    ok = ok && P::good(P::key(pv));
    const R inv = rcp<R>(pv);
    w[42] = inv;
  }
  {  // pivot 13: state 21 (X_ac), 3 rows x 2 cols
    const R pv = w[58];
    const typename P::K cm = P::kmax(P::kmax(P::key(w[89]), P::key(w[116])), P::key(w[148]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[58] = inv;
    { const R l = w[89] * inv; w[89] = l;
      w[97] -= l * w[59];
      w[102] -= l * w[60];
    }
    { const R l = w[116] * inv; w[116] = l;
      w[124] -= l * w[59];
      w[129] -= l * w[60];
    }
    { const R l = w[148] * inv; w[148] = l;
      w[156] -= l * w[59];
      w[161] -= l * w[60];
    }
  }
  {  // pivot 14: state 18 (X_fa), 4 rows x 2 cols
    const R pv = w[61];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::key(w[65]), P::key(w[90])), P::key(w[117])), P::key(w[149]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[61] = inv;
    { const R l = w[65] * inv; w[65] = l;
      w[66] -= l * w[62];
      w[68] -= l * w[63];
    }
    { const R l = w[90] * inv; w[90] = l;
      w[91] -= l * w[62];
      w[102] -= l * w[63];
    }
    { const R l = w[117] * inv; w[117] = l;
      w[118] -= l * w[62];
      w[129] -= l * w[63];
    }
    { const R l = w[149] * inv; w[149] = l;
      w[150] -= l * w[62];
      w[161] -= l * w[63];
    }
  }
  {  // pivot 15: state 2 (S_fa), 3 rows x 2 cols
    const R pv = w[66];
    const typename P::K cm = P::kmax(P::kmax(P::key(w[91]), P::key(w[118])), P::key(w[150]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[66] = inv;
    { const R l = w[91] * inv; w[91] = l;
      w[99] -= l * w[67];
      w[102] -= l * w[68];
    }
    { const R l = w[118] * inv; w[118] = l;
      w[126] -= l * w[67];
      w[129] -= l * w[68];
    }
    { const R l = w[150] * inv; w[150] = l;
      w[158] -= l * w[67];
      w[161] -= l * w[68];
    }
  }
  {  // pivot 16: state 20 (X_pro), 4 rows x 2 cols
    const R pv = w[69];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::key(w[92]), P::key(w[104])), P::key(w[119])), P::key(w[151]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[69] = inv;
    { const R l = w[92] * inv; w[92] = l;
      w[98] -= l * w[70];
      w[102] -= l * w[71];
    }
    { const R l = w[104] * inv; w[104] = l;
      w[109] -= l * w[70];
      w[113] -= l * w[71];
    }
    { const R l = w[119] * inv; w[119] = l;
      w[125] -= l * w[70];
      w[129] -= l * w[71];
    }
    { const R l = w[151] * inv; w[151] = l;
      w[157] -= l * w[70];
      w[161] -= l * w[71];
    }
  }
  {  // pivot 17: state 16 (X_su), 6 rows x 2 cols
    const R pv = w[72];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::kmax(P::kmax(P::key(w[77]), P::key(w[93])), P::key(w[105])), P::key(w[120])), P::key(w[138])), P::key(w[152]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[72] = inv;
    { const R l = w[77] * inv; w[77] = l;
      w[78] -= l * w[73];
      w[80] -= l * w[74];
    }
    { const R l = w[93] * inv; w[93] = l;
      w[94] -= l * w[73];
      w[102] -= l * w[74];
    }
    { const R l = w[105] * inv; w[105] = l;
      w[106] -= l * w[73];
      w[113] -= l * w[74];
    }
    { const R l = w[120] * inv; w[120] = l;
      w[121] -= l * w[73];
      w[129] -= l * w[74];
    }
    { const R l = w[138] * inv; w[138] = l;
      w[139] -= l * w[73];
      w[145] -= l * w[74];
    }
    { const R l = w[152] * inv; w[152] = l;
      w[153] -= l * w[73];
      w[161] -= l * w[74];
    }
  }
  {  // pivot 18: state 0 (S_su), 5 rows x 2 cols
    const R pv = w[78];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::kmax(P::key(w[94]), P::key(w[106])), P::key(w[121])), P::key(w[139])), P::key(w[153]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[78] = inv;
    { const R l = w[94] * inv; w[94] = l;
      w[99] -= l * w[79];
      w[102] -= l * w[80];
    }
    { const R l = w[106] * inv; w[106] = l;
      w[110] -= l * w[79];
      w[113] -= l * w[80];
    }
    { const R l = w[121] * inv; w[121] = l;
      w[126] -= l * w[79];
      w[129] -= l * w[80];
    }
    { const R l = w[139] * inv; w[139] = l;
      w[142] -= l * w[79];
      w[145] -= l * w[80];
    }
    { const R l = w[153] * inv; w[153] = l;
      w[158] -= l * w[79];
      w[161] -= l * w[80];
    }
  }
  {  // pivot 19: state 17 (X_aa), 7 rows x 2 cols
    const R pv = w[81];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::kmax(P::kmax(P::kmax(P::key(w[85]), P::key(w[95])), P::key(w[107])), P::key(w[122])), P::key(w[131])), P::key(w[140])), P::key(w[154]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[81] = inv;
    { const R l = w[85] * inv; w[85] = l;
      w[86] -= l * w[82];
      w[88] -= l * w[83];
    }
    { const R l = w[95] * inv; w[95] = l;
      w[96] -= l * w[82];
      w[102] -= l * w[83];
    }
    { const R l = w[107] * inv; w[107] = l;
      w[108] -= l * w[82];
      w[113] -= l * w[83];
    }
    { const R l = w[122] * inv; w[122] = l;
      w[123] -= l * w[82];
      w[129] -= l * w[83];
    }
    { const R l = w[131] * inv; w[131] = l;
      w[132] -= l * w[82];
      w[136] -= l * w[83];
    }
    { const R l = w[140] * inv; w[140] = l;
      w[141] -= l * w[82];
      w[145] -= l * w[83];
    }
    { const R l = w[154] * inv; w[154] = l;
      w[155] -= l * w[82];
      w[161] -= l * w[83];
    }
  }
  {  // pivot 20: state 1 (S_aa), 6 rows x 2 cols
    const R pv = w[86];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::kmax(P::kmax(P::key(w[96]), P::key(w[108])), P::key(w[123])), P::key(w[132])), P::key(w[141])), P::key(w[155]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[86] = inv;
    { const R l = w[96] * inv; w[96] = l;
      w[99] -= l * w[87];
      w[102] -= l * w[88];
    }
    { const R l = w[108] * inv; w[108] = l;
      w[110] -= l * w[87];
      w[113] -= l * w[88];
    }
    { const R l = w[123] * inv; w[123] = l;
      w[126] -= l * w[87];
      w[129] -= l * w[88];
    }
    { const R l = w[132] * inv; w[132] = l;
      w[133] -= l * w[87];
      w[136] -= l * w[88];
    }
    { const R l = w[141] * inv; w[141] = l;
      w[142] -= l * w[87];
      w[145] -= l * w[88];
    }
    { const R l = w[155] * inv; w[155] = l;
      w[158] -= l * w[87];
      w[161] -= l * w[88];
    }
  }
  {  // pivot 21: state 6 (S_ac), 2 rows x 6 cols
    const R pv = w[97];
    const typename P::K cm = P::kmax(P::key(w[124]), P::key(w[156]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[97] = inv;
    { const R l = w[124] * inv; w[124] = l;
      w[125] -= l * w[98];
      w[126] -= l * w[99];
      w[127] -= l * w[100];
      w[128] -= l * w[101];
      w[129] -= l * w[102];
      w[130] -= l * w[103];
    }
    { const R l = w[156] * inv; w[156] = l;
      w[157] -= l * w[98];
      w[158] -= l * w[99];
      w[159] -= l * w[100];
      w[160] -= l * w[101];
      w[161] -= l * w[102];
      w[162] -= l * w[103];
    }
  }
  {  // pivot 22: state 5 (S_pro), 2 rows x 5 cols
    const R pv = w[109];
    const typename P::K cm = P::kmax(P::key(w[125]), P::key(w[157]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[109] = inv;
    { const R l = w[125] * inv; w[125] = l;
      w[126] -= l * w[110];
      w[127] -= l * w[111];
      w[128] -= l * w[112];
      w[129] -= l * w[113];
      w[130] -= l * w[114];
    }
    { const R l = w[157] * inv; w[157] = l;
      w[158] -= l * w[110];
      w[159] -= l * w[111];
      w[160] -= l * w[112];
      w[161] -= l * w[113];
      w[162] -= l * w[114];
    }
  }
  {  // pivot 23: state 12 (X_c), 3 rows x 4 cols
    const R pv = w[126];
    const typename P::K cm = P::kmax(P::kmax(P::key(w[133]), P::key(w[142])), P::key(w[158]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[126] = inv;
    { const R l = w[133] * inv; w[133] = l;
      w[134] -= l * w[127];
      w[135] -= l * w[128];
      w[136] -= l * w[129];
      w[137] -= l * w[130];
    }
    { const R l = w[142] * inv; w[142] = l;
      w[143] -= l * w[127];
      w[144] -= l * w[128];
      w[145] -= l * w[129];
      w[146] -= l * w[130];
    }
    { const R l = w[158] * inv; w[158] = l;
      w[159] -= l * w[127];
      w[160] -= l * w[128];
      w[161] -= l * w[129];
      w[162] -= l * w[130];
    }
  }
  {  // pivot 24: state 3 (S_va), 3 rows x 3 cols
    const R pv = w[134];
    const typename P::K cm = P::kmax(P::kmax(P::key(w[143]), P::key(w[159])), P::key(w[163]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[134] = inv;
    { const R l = w[143] * inv; w[143] = l;
      w[144] -= l * w[135];
      w[145] -= l * w[136];
      w[146] -= l * w[137];
    }
    { const R l = w[159] * inv; w[159] = l;
      w[160] -= l * w[135];
      w[161] -= l * w[136];
      w[162] -= l * w[137];
    }
    { const R l = w[163] * inv; w[163] = l;
      w[164] -= l * w[135];
      w[165] -= l * w[136];
      w[166] -= l * w[137];
    }
  }
  {  // pivot 25: state 4 (S_bu), 2 rows x 2 cols
    const R pv = w[144];
    const typename P::K cm = P::kmax(P::key(w[160]), P::key(w[164]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[144] = inv;
    { const R l = w[160] * inv; w[160] = l;
      w[161] -= l * w[145];
      w[162] -= l * w[146];
    }
    { const R l = w[164] * inv; w[164] = l;
      w[165] -= l * w[145];
      w[166] -= l * w[146];
    }
  }
  {  // pivot 26: state 10 (S_IN), 1 rows x 1 cols
    const R pv = w[161];
    const typename P::K cm = P::key(w[165]);
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[161] = inv;
    { const R l = w[165] * inv; w[165] = l;
      w[166] -= l * w[162];
    }
  }
  {  // pivot 27: state 19 (X_c4), 0 rows x 0 cols
    const R pv = w[166];
    ok = ok && P::good(P::key(pv));
    const R inv = rcp<R>(pv);
    w[166] = inv;
  }
  return ok;
}

// Solve W x = b in place (b indexed by state; b[S_h2] is left as it is:
// W_d's S_h2 row is the identity's).
template <class R, class W>
CHAD_HD void solve(W w, R* b) {
  R z0 = b[11];
  R z1 = b[23];
  R z2 = b[24];
  R z3 = b[25];
  R z4 = b[13];
  R z5 = b[14];
  R z6 = b[15];
  R z7 = b[22];
  R z8 = b[8];
  R z9 = b[26];
  R z10 = b[27];
  R z11 = b[28];
  R z12 = b[9];
  R z13 = b[21];
  R z14 = b[18];
  R z15 = b[2];
  R z16 = b[20];
  R z17 = b[16];
  R z18 = b[0];
  R z19 = b[17];
  R z20 = b[1];
  R z21 = b[6];
  R z22 = b[5];
  R z23 = b[12];
  R z24 = b[3];
  R z25 = b[4];
  R z26 = b[10];
  R z27 = b[19];
  z8 -= w[14] * z7;
  z10 -= w[23] * z8;
  z10 -= w[24] * z9;
  z11 -= w[30] * z9;
  z11 -= w[31] * z10;
  z12 -= w[37] * z4;
  z12 -= w[38] * z5;
  z12 -= w[39] * z6;
  z12 -= w[40] * z7;
  z12 -= w[41] * z11;
  z15 -= w[64] * z6;
  z15 -= w[65] * z14;
  z18 -= w[75] * z4;
  z18 -= w[76] * z6;
  z18 -= w[77] * z17;
  z20 -= w[84] * z5;
  z20 -= w[85] * z19;
  z21 -= w[89] * z13;
  z21 -= w[90] * z14;
  z21 -= w[91] * z15;
  z21 -= w[92] * z16;
  z21 -= w[93] * z17;
  z21 -= w[94] * z18;
  z21 -= w[95] * z19;
  z21 -= w[96] * z20;
  z22 -= w[104] * z16;
  z22 -= w[105] * z17;
  z22 -= w[106] * z18;
  z22 -= w[107] * z19;
  z22 -= w[108] * z20;
  z23 -= w[115] * z7;
  z23 -= w[116] * z13;
  z23 -= w[117] * z14;
  z23 -= w[118] * z15;
  z23 -= w[119] * z16;
  z23 -= w[120] * z17;
  z23 -= w[121] * z18;
  z23 -= w[122] * z19;
  z23 -= w[123] * z20;
  z23 -= w[124] * z21;
  z23 -= w[125] * z22;
  z24 -= w[131] * z19;
  z24 -= w[132] * z20;
  z24 -= w[133] * z23;
  z25 -= w[138] * z17;
  z25 -= w[139] * z18;
  z25 -= w[140] * z19;
  z25 -= w[141] * z20;
  z25 -= w[142] * z23;
  z25 -= w[143] * z24;
  z26 -= w[147] * z7;
  z26 -= w[148] * z13;
  z26 -= w[149] * z14;
  z26 -= w[150] * z15;
  z26 -= w[151] * z16;
  z26 -= w[152] * z17;
  z26 -= w[153] * z18;
  z26 -= w[154] * z19;
  z26 -= w[155] * z20;
  z26 -= w[156] * z21;
  z26 -= w[157] * z22;
  z26 -= w[158] * z23;
  z26 -= w[159] * z24;
  z26 -= w[160] * z25;
  z27 -= w[163] * z24;
  z27 -= w[164] * z25;
  z27 -= w[165] * z26;
  z27 *= w[166];
  z26 -= w[162] * z27;
  z26 *= w[161];
  z25 -= w[145] * z26;
  z25 -= w[146] * z27;
  z25 *= w[144];
  z24 -= w[135] * z25;
  z24 -= w[136] * z26;
  z24 -= w[137] * z27;
  z24 *= w[134];
  z23 -= w[127] * z24;
  z23 -= w[128] * z25;
  z23 -= w[129] * z26;
  z23 -= w[130] * z27;
  z23 *= w[126];
  z22 -= w[110] * z23;
  z22 -= w[111] * z24;
  z22 -= w[112] * z25;
  z22 -= w[113] * z26;
  z22 -= w[114] * z27;
  z22 *= w[109];
  z21 -= w[98] * z22;
  z21 -= w[99] * z23;
  z21 -= w[100] * z24;
  z21 -= w[101] * z25;
  z21 -= w[102] * z26;
  z21 -= w[103] * z27;
  z21 *= w[97];
  z20 -= w[87] * z23;
  z20 -= w[88] * z26;
  z20 *= w[86];
  z19 -= w[82] * z20;
  z19 -= w[83] * z26;
  z19 *= w[81];
  z18 -= w[79] * z23;
  z18 -= w[80] * z26;
  z18 *= w[78];
  z17 -= w[73] * z18;
  z17 -= w[74] * z26;
  z17 *= w[72];
  z16 -= w[70] * z22;
  z16 -= w[71] * z26;
  z16 *= w[69];
  z15 -= w[67] * z23;
  z15 -= w[68] * z26;
  z15 *= w[66];
  z14 -= w[62] * z15;
  z14 -= w[63] * z26;
  z14 *= w[61];
  z13 -= w[59] * z21;
  z13 -= w[60] * z26;
  z13 *= w[58];
  z12 -= w[43] * z13;
  z12 -= w[44] * z14;
  z12 -= w[45] * z15;
  z12 -= w[46] * z16;
  z12 -= w[47] * z17;
  z12 -= w[48] * z18;
  z12 -= w[49] * z19;
  z12 -= w[50] * z20;
  z12 -= w[51] * z21;
  z12 -= w[52] * z22;
  z12 -= w[53] * z23;
  z12 -= w[54] * z24;
  z12 -= w[55] * z25;
  z12 -= w[56] * z26;
  z12 -= w[57] * z27;
  z12 *= w[42];
  z11 -= w[33] * z12;
  z11 -= w[34] * z13;
  z11 -= w[35] * z21;
  z11 -= w[36] * z26;
  z11 *= w[32];
  z10 -= w[26] * z11;
  z10 -= w[27] * z13;
  z10 -= w[28] * z21;
  z10 -= w[29] * z26;
  z10 *= w[25];
  z9 -= w[21] * z10;
  z9 -= w[22] * z11;
  z9 *= w[20];
  z8 -= w[16] * z10;
  z8 -= w[17] * z13;
  z8 -= w[18] * z21;
  z8 -= w[19] * z26;
  z8 *= w[15];
  z7 -= w[13] * z26;
  z7 *= w[12];
  z6 -= w[11] * z23;
  z6 *= w[10];
  z5 -= w[9] * z23;
  z5 *= w[8];
  z4 -= w[7] * z23;
  z4 *= w[6];
  z3 *= w[5];
  z2 *= w[4];
  z1 -= w[3] * z23;
  z1 *= w[2];
  z0 -= w[1] * z23;
  z0 *= w[0];
  b[11] = z0;
  b[23] = z1;
  b[24] = z2;
  b[25] = z3;
  b[13] = z4;
  b[14] = z5;
  b[15] = z6;
  b[22] = z7;
  b[8] = z8;
  b[26] = z9;
  b[27] = z10;
  b[28] = z11;
  b[9] = z12;
  b[21] = z13;
  b[18] = z14;
  b[2] = z15;
  b[20] = z16;
  b[16] = z17;
  b[0] = z18;
  b[17] = z19;
  b[1] = z20;
  b[6] = z21;
  b[5] = z22;
  b[12] = z23;
  b[3] = z24;
  b[4] = z25;
  b[10] = z26;
  b[19] = z27;
}

constexpr int kFactorFlops = 397;
constexpr int kSolveFlops = 306;

// The LU as a type, so that the kernels can take it as a template parameter.
struct Lu {
  using Index = Idx;
  static constexpr int nnz = kNNZ;
  static constexpr int store = kStore;
  template <class R, class W>
  static CHAD_HD void form(W w, R g) { form_w<R>(w, g); }
  template <class R, class W>
  static CHAD_HD bool lu(W w) { return factor<R>(w); }
  template <class R, class W>
  static CHAD_HD void sub(W w, R* b) { solve<R>(w, b); }
};

}  // namespace spa
}  // namespace chad
