// GENERATED by gen_sparse.py from the library's own Jacobian pattern -- do not edit.
// Static-order (Markowitz) sparse LU of W_d = I - g J_d for the 29 ADM1 states
// (J_d: the Jacobian with S_H held fixed).
// pattern nnz(J_d) = 174, slots with fill = 203
#pragma once
#include "adm1_device.cuh"

namespace chad {
namespace sp {

constexpr int kNNZ = 203;
constexpr int kNNZ_J = 174;
constexpr int kPiv = 29;
constexpr int kStore = 203;
// elimination position -> state index
constexpr int kOrder[kPiv] = {11, 23, 24, 25, 13, 14, 15, 8, 26, 28, 21, 22, 27, 9, 16, 0, 18, 2, 20, 17, 1, 6, 5, 12, 3, 4, 7, 10, 19};

CHAD_HD constexpr int slot(int r, int c) {
  // row-major table over states, -1 = structurally zero
  const int t[NS * NS] = {
      73, -1, -1, -1, -1, -1, -1, -1, -1, -1, 75, -1, 74, 70, -1, 71, 72, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, 95, -1, -1, -1, -1, -1, -1, -1, -1, 97, -1, 96, -1, 93, -1, -1, 94, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, 82, -1, -1, -1, -1, 84, -1, -1, 85, -1, 83, -1, -1, 80, -1, -1, 81, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, 144, -1, 146, 147, -1, -1, 148, -1, -1, 149, -1, 145, -1, -1, -1, -1, 143, -1, 150, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      152, 154, -1, 156, 157, -1, -1, 158, -1, -1, 159, -1, 155, -1, -1, -1, 151, 153, -1, 160, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      115, 118, -1, 121, 122, 119, -1, 123, -1, -1, 124, -1, 120, -1, -1, -1, 114, 117, -1, 125, 116, -1, -1, -1, -1, -1, -1, -1, -1,
      100, 105, 102, 109, 110, 107, 106, 111, -1, -1, 112, -1, 108, -1, -1, -1, 99, 104, 101, 113, 103, 98, -1, -1, -1, -1, -1, -1, -1,
      167, 172, 169, 176, 177, 174, 173, 178, -1, 165, 179, -1, 175, -1, -1, -1, 166, 171, 168, 180, 170, -1, 163, -1, -1, -1, 161, 164, 162,
      -1, -1, -1, -1, -1, -1, 16, 17, 12, -1, 18, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 13, 14, -1, -1, -1, -1, 15, -1,
      53, 58, 55, 62, 63, 60, 59, 64, -1, 51, 65, -1, 61, 44, 45, 46, 52, 57, 54, 66, 56, 48, 49, -1, -1, -1, -1, 50, 47,
      184, 189, 186, 193, 194, 191, 190, 195, -1, -1, 196, -1, 192, -1, -1, -1, 183, 188, 185, 197, 187, 181, 182, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 0, 1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      129, 134, 131, 138, 139, 136, 135, 140, -1, -1, 141, -1, 137, -1, -1, -1, 128, 133, 130, 142, 132, 126, 127, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 7, 6, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 9, -1, 8, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 11, -1, -1, 10, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      68, -1, -1, -1, -1, -1, -1, -1, -1, -1, 69, -1, -1, -1, -1, -1, 67, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, 91, -1, -1, -1, -1, -1, -1, -1, -1, 92, -1, -1, -1, -1, -1, -1, 90, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, 77, -1, -1, -1, -1, 78, -1, -1, 79, -1, -1, -1, -1, -1, -1, -1, 76, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, 198, 199, -1, -1, 200, -1, -1, 201, -1, -1, -1, -1, -1, -1, -1, -1, 202, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, 87, -1, 88, -1, -1, 89, -1, -1, -1, -1, -1, -1, -1, -1, -1, 86, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, 29, -1, -1, -1, 30, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 28, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, 32, -1, -1, 33, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 31, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 3, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 2, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 4, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 5, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, 22, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 19, 21, 20,
      -1, -1, -1, -1, -1, -1, 41, 42, 34, 40, 43, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 37, 38, -1, -1, -1, 35, 39, 36,
      -1, -1, -1, -1, -1, -1, -1, 27, -1, 26, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 23, 25, 24
  };
  return t[r * NS + c];
}

struct Idx {
  static CHAD_HD constexpr int at(int r, int c) { return slot(r, c); }
  static constexpr int size = kStore;
};

// diagonal slots in elimination order
constexpr int kDiag[kPiv] = {0, 2, 4, 5, 6, 8, 10, 12, 19, 24, 28, 31, 39, 51, 67, 73, 76, 82, 86, 90, 95, 106, 119, 137, 146, 157, 178, 196, 202};

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
  w[19] += R(1);
  w[24] += R(1);
  w[28] += R(1);
  w[31] += R(1);
  w[39] += R(1);
  w[51] += R(1);
  w[67] += R(1);
  w[73] += R(1);
  w[76] += R(1);
  w[82] += R(1);
  w[86] += R(1);
  w[90] += R(1);
  w[95] += R(1);
  w[106] += R(1);
  w[119] += R(1);
  w[137] += R(1);
  w[146] += R(1);
  w[157] += R(1);
  w[178] += R(1);
  w[196] += R(1);
  w[202] += R(1);
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
    const typename P::K cm = P::kmax(P::key(w[44]), P::key(w[70]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[6] = inv;
    { const R l = w[44] * inv; w[44] = l;
      w[61] -= l * w[7];
    }
    { const R l = w[70] * inv; w[70] = l;
      w[74] -= l * w[7];
    }
  }
  {  // pivot 5: state 14 (X_pr), 2 rows x 1 cols
    const R pv = w[8];
    const typename P::K cm = P::kmax(P::key(w[45]), P::key(w[93]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[8] = inv;
    { const R l = w[45] * inv; w[45] = l;
      w[61] -= l * w[9];
    }
    { const R l = w[93] * inv; w[93] = l;
      w[96] -= l * w[9];
    }
  }
  {  // pivot 6: state 15 (X_li), 3 rows x 1 cols
    const R pv = w[10];
    const typename P::K cm = P::kmax(P::kmax(P::key(w[46]), P::key(w[71])), P::key(w[80]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[10] = inv;
    { const R l = w[46] * inv; w[46] = l;
      w[61] -= l * w[11];
    }
    { const R l = w[71] * inv; w[71] = l;
      w[74] -= l * w[11];
    }
    { const R l = w[80] * inv; w[80] = l;
      w[83] -= l * w[11];
    }
  }
  {  // pivot 7: state 8 (S_ch4), 1 rows x 6 cols
    const R pv = w[12];
    const typename P::K cm = P::key(w[34]);
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[12] = inv;
    { const R l = w[34] * inv; w[34] = l;
      w[37] -= l * w[13];
      w[38] -= l * w[14];
      w[39] -= l * w[15];
      w[41] -= l * w[16];
      w[42] -= l * w[17];
      w[43] -= l * w[18];
    }
  }
  {  // pivot 8: state 26 (S_gas_h2), 3 rows x 3 cols
    const R pv = w[19];
    const typename P::K cm = P::kmax(P::kmax(P::key(w[23]), P::key(w[35])), P::key(w[161]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[19] = inv;
    { const R l = w[23] * inv; w[23] = l;
      w[24] -= l * w[20];
      w[25] -= l * w[21];
      w[27] -= l * w[22];
    }
    { const R l = w[35] * inv; w[35] = l;
      w[36] -= l * w[20];
      w[39] -= l * w[21];
      w[42] -= l * w[22];
    }
    { const R l = w[161] * inv; w[161] = l;
      w[162] -= l * w[20];
      w[164] -= l * w[21];
      w[178] -= l * w[22];
    }
  }
  {  // pivot 9: state 28 (S_gas_co2), 3 rows x 3 cols
    const R pv = w[24];
    const typename P::K cm = P::kmax(P::kmax(P::key(w[36]), P::key(w[47])), P::key(w[162]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[24] = inv;
    { const R l = w[36] * inv; w[36] = l;
      w[39] -= l * w[25];
      w[40] -= l * w[26];
      w[42] -= l * w[27];
    }
    { const R l = w[47] * inv; w[47] = l;
      w[50] -= l * w[25];
      w[51] -= l * w[26];
      w[64] -= l * w[27];
    }
    { const R l = w[162] * inv; w[162] = l;
      w[164] -= l * w[25];
      w[165] -= l * w[26];
      w[178] -= l * w[27];
    }
  }
  {  // pivot 10: state 21 (X_ac), 5 rows x 2 cols
    const R pv = w[28];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::kmax(P::key(w[37]), P::key(w[48])), P::key(w[98])), P::key(w[126])), P::key(w[181]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[28] = inv;
    { const R l = w[37] * inv; w[37] = l;
      w[41] -= l * w[29];
      w[43] -= l * w[30];
    }
    { const R l = w[48] * inv; w[48] = l;
      w[59] -= l * w[29];
      w[65] -= l * w[30];
    }
    { const R l = w[98] * inv; w[98] = l;
      w[106] -= l * w[29];
      w[112] -= l * w[30];
    }
    { const R l = w[126] * inv; w[126] = l;
      w[135] -= l * w[29];
      w[141] -= l * w[30];
    }
    { const R l = w[181] * inv; w[181] = l;
      w[190] -= l * w[29];
      w[196] -= l * w[30];
    }
  }
  {  // pivot 11: state 22 (X_h2), 5 rows x 2 cols
    const R pv = w[31];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::kmax(P::key(w[38]), P::key(w[49])), P::key(w[127])), P::key(w[163])), P::key(w[182]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[31] = inv;
    { const R l = w[38] * inv; w[38] = l;
      w[42] -= l * w[32];
      w[43] -= l * w[33];
    }
    { const R l = w[49] * inv; w[49] = l;
      w[64] -= l * w[32];
      w[65] -= l * w[33];
    }
    { const R l = w[127] * inv; w[127] = l;
      w[140] -= l * w[32];
      w[141] -= l * w[33];
    }
    { const R l = w[163] * inv; w[163] = l;
      w[178] -= l * w[32];
      w[179] -= l * w[33];
    }
    { const R l = w[182] * inv; w[182] = l;
      w[195] -= l * w[32];
      w[196] -= l * w[33];
    }
  }
  {  // pivot 12: state 27 (S_gas_ch4), 2 rows x 4 cols
    const R pv = w[39];
    const typename P::K cm = P::kmax(P::key(w[50]), P::key(w[164]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[39] = inv;
    { const R l = w[50] * inv; w[50] = l;
      w[51] -= l * w[40];
      w[59] -= l * w[41];
      w[64] -= l * w[42];
      w[65] -= l * w[43];
    }
    { const R l = w[164] * inv; w[164] = l;
      w[165] -= l * w[40];
      w[173] -= l * w[41];
      w[178] -= l * w[42];
      w[179] -= l * w[43];
    }
  }
  {  // pivot 13: state 9 (S_IC), 1 rows x 15 cols
    const R pv = w[51];
    const typename P::K cm = P::key(w[165]);
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[51] = inv;
    { const R l = w[165] * inv; w[165] = l;
      w[166] -= l * w[52];
      w[167] -= l * w[53];
      w[168] -= l * w[54];
      w[169] -= l * w[55];
      w[170] -= l * w[56];
      w[171] -= l * w[57];
      w[172] -= l * w[58];
      w[173] -= l * w[59];
      w[174] -= l * w[60];
      w[175] -= l * w[61];
      w[176] -= l * w[62];
      w[177] -= l * w[63];
      w[178] -= l * w[64];
      w[179] -= l * w[65];
      w[180] -= l * w[66];
    }
  }
  {  // pivot 14: state 16 (X_su), 7 rows x 2 cols
    const R pv = w[67];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::kmax(P::kmax(P::kmax(P::key(w[72]), P::key(w[99])), P::key(w[114])), P::key(w[128])), P::key(w[151])), P::key(w[166])), P::key(w[183]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[67] = inv;
    { const R l = w[72] * inv; w[72] = l;
      w[73] -= l * w[68];
      w[75] -= l * w[69];
    }
    { const R l = w[99] * inv; w[99] = l;
      w[100] -= l * w[68];
      w[112] -= l * w[69];
    }
    { const R l = w[114] * inv; w[114] = l;
      w[115] -= l * w[68];
      w[124] -= l * w[69];
    }
    { const R l = w[128] * inv; w[128] = l;
      w[129] -= l * w[68];
      w[141] -= l * w[69];
    }
    { const R l = w[151] * inv; w[151] = l;
      w[152] -= l * w[68];
      w[159] -= l * w[69];
    }
    { const R l = w[166] * inv; w[166] = l;
      w[167] -= l * w[68];
      w[179] -= l * w[69];
    }
    { const R l = w[183] * inv; w[183] = l;
      w[184] -= l * w[68];
      w[196] -= l * w[69];
    }
  }
  {  // pivot 15: state 0 (S_su), 6 rows x 2 cols
    const R pv = w[73];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::kmax(P::kmax(P::key(w[100]), P::key(w[115])), P::key(w[129])), P::key(w[152])), P::key(w[167])), P::key(w[184]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[73] = inv;
    { const R l = w[100] * inv; w[100] = l;
      w[108] -= l * w[74];
      w[112] -= l * w[75];
    }
    { const R l = w[115] * inv; w[115] = l;
      w[120] -= l * w[74];
      w[124] -= l * w[75];
    }
    { const R l = w[129] * inv; w[129] = l;
      w[137] -= l * w[74];
      w[141] -= l * w[75];
    }
    { const R l = w[152] * inv; w[152] = l;
      w[155] -= l * w[74];
      w[159] -= l * w[75];
    }
    { const R l = w[167] * inv; w[167] = l;
      w[175] -= l * w[74];
      w[179] -= l * w[75];
    }
    { const R l = w[184] * inv; w[184] = l;
      w[192] -= l * w[74];
      w[196] -= l * w[75];
    }
  }
  {  // pivot 16: state 18 (X_fa), 5 rows x 3 cols
    const R pv = w[76];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::kmax(P::key(w[81]), P::key(w[101])), P::key(w[130])), P::key(w[168])), P::key(w[185]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[76] = inv;
    { const R l = w[81] * inv; w[81] = l;
      w[82] -= l * w[77];
      w[84] -= l * w[78];
      w[85] -= l * w[79];
    }
    { const R l = w[101] * inv; w[101] = l;
      w[102] -= l * w[77];
      w[111] -= l * w[78];
      w[112] -= l * w[79];
    }
    { const R l = w[130] * inv; w[130] = l;
      w[131] -= l * w[77];
      w[140] -= l * w[78];
      w[141] -= l * w[79];
    }
    { const R l = w[168] * inv; w[168] = l;
      w[169] -= l * w[77];
      w[178] -= l * w[78];
      w[179] -= l * w[79];
    }
    { const R l = w[185] * inv; w[185] = l;
      w[186] -= l * w[77];
      w[195] -= l * w[78];
      w[196] -= l * w[79];
    }
  }
  {  // pivot 17: state 2 (S_fa), 4 rows x 3 cols
    const R pv = w[82];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::key(w[102]), P::key(w[131])), P::key(w[169])), P::key(w[186]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[82] = inv;
    { const R l = w[102] * inv; w[102] = l;
      w[108] -= l * w[83];
      w[111] -= l * w[84];
      w[112] -= l * w[85];
    }
    { const R l = w[131] * inv; w[131] = l;
      w[137] -= l * w[83];
      w[140] -= l * w[84];
      w[141] -= l * w[85];
    }
    { const R l = w[169] * inv; w[169] = l;
      w[175] -= l * w[83];
      w[178] -= l * w[84];
      w[179] -= l * w[85];
    }
    { const R l = w[186] * inv; w[186] = l;
      w[192] -= l * w[83];
      w[195] -= l * w[84];
      w[196] -= l * w[85];
    }
  }
  {  // pivot 18: state 20 (X_pro), 5 rows x 3 cols
    const R pv = w[86];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::kmax(P::key(w[103]), P::key(w[116])), P::key(w[132])), P::key(w[170])), P::key(w[187]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[86] = inv;
    { const R l = w[103] * inv; w[103] = l;
      w[107] -= l * w[87];
      w[111] -= l * w[88];
      w[112] -= l * w[89];
    }
    { const R l = w[116] * inv; w[116] = l;
      w[119] -= l * w[87];
      w[123] -= l * w[88];
      w[124] -= l * w[89];
    }
    { const R l = w[132] * inv; w[132] = l;
      w[136] -= l * w[87];
      w[140] -= l * w[88];
      w[141] -= l * w[89];
    }
    { const R l = w[170] * inv; w[170] = l;
      w[174] -= l * w[87];
      w[178] -= l * w[88];
      w[179] -= l * w[89];
    }
    { const R l = w[187] * inv; w[187] = l;
      w[191] -= l * w[87];
      w[195] -= l * w[88];
      w[196] -= l * w[89];
    }
  }
  {  // pivot 19: state 17 (X_aa), 8 rows x 2 cols
    const R pv = w[90];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::kmax(P::kmax(P::kmax(P::kmax(P::key(w[94]), P::key(w[104])), P::key(w[117])), P::key(w[133])), P::key(w[143])), P::key(w[153])), P::key(w[171])), P::key(w[188]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[90] = inv;
    { const R l = w[94] * inv; w[94] = l;
      w[95] -= l * w[91];
      w[97] -= l * w[92];
    }
    { const R l = w[104] * inv; w[104] = l;
      w[105] -= l * w[91];
      w[112] -= l * w[92];
    }
    { const R l = w[117] * inv; w[117] = l;
      w[118] -= l * w[91];
      w[124] -= l * w[92];
    }
    { const R l = w[133] * inv; w[133] = l;
      w[134] -= l * w[91];
      w[141] -= l * w[92];
    }
    { const R l = w[143] * inv; w[143] = l;
      w[144] -= l * w[91];
      w[149] -= l * w[92];
    }
    { const R l = w[153] * inv; w[153] = l;
      w[154] -= l * w[91];
      w[159] -= l * w[92];
    }
    { const R l = w[171] * inv; w[171] = l;
      w[172] -= l * w[91];
      w[179] -= l * w[92];
    }
    { const R l = w[188] * inv; w[188] = l;
      w[189] -= l * w[91];
      w[196] -= l * w[92];
    }
  }
  {  // pivot 20: state 1 (S_aa), 7 rows x 2 cols
    const R pv = w[95];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::kmax(P::kmax(P::kmax(P::key(w[105]), P::key(w[118])), P::key(w[134])), P::key(w[144])), P::key(w[154])), P::key(w[172])), P::key(w[189]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[95] = inv;
    { const R l = w[105] * inv; w[105] = l;
      w[108] -= l * w[96];
      w[112] -= l * w[97];
    }
    { const R l = w[118] * inv; w[118] = l;
      w[120] -= l * w[96];
      w[124] -= l * w[97];
    }
    { const R l = w[134] * inv; w[134] = l;
      w[137] -= l * w[96];
      w[141] -= l * w[97];
    }
    { const R l = w[144] * inv; w[144] = l;
      w[145] -= l * w[96];
      w[149] -= l * w[97];
    }
    { const R l = w[154] * inv; w[154] = l;
      w[155] -= l * w[96];
      w[159] -= l * w[97];
    }
    { const R l = w[172] * inv; w[172] = l;
      w[175] -= l * w[96];
      w[179] -= l * w[97];
    }
    { const R l = w[189] * inv; w[189] = l;
      w[192] -= l * w[96];
      w[196] -= l * w[97];
    }
  }
  {  // pivot 21: state 6 (S_ac), 3 rows x 7 cols
    const R pv = w[106];
    const typename P::K cm = P::kmax(P::kmax(P::key(w[135]), P::key(w[173])), P::key(w[190]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[106] = inv;
    { const R l = w[135] * inv; w[135] = l;
      w[136] -= l * w[107];
      w[137] -= l * w[108];
      w[138] -= l * w[109];
      w[139] -= l * w[110];
      w[140] -= l * w[111];
      w[141] -= l * w[112];
      w[142] -= l * w[113];
    }
    { const R l = w[173] * inv; w[173] = l;
      w[174] -= l * w[107];
      w[175] -= l * w[108];
      w[176] -= l * w[109];
      w[177] -= l * w[110];
      w[178] -= l * w[111];
      w[179] -= l * w[112];
      w[180] -= l * w[113];
    }
    { const R l = w[190] * inv; w[190] = l;
      w[191] -= l * w[107];
      w[192] -= l * w[108];
      w[193] -= l * w[109];
      w[194] -= l * w[110];
      w[195] -= l * w[111];
      w[196] -= l * w[112];
      w[197] -= l * w[113];
    }
  }
  {  // pivot 22: state 5 (S_pro), 3 rows x 6 cols
    const R pv = w[119];
    const typename P::K cm = P::kmax(P::kmax(P::key(w[136]), P::key(w[174])), P::key(w[191]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[119] = inv;
    { const R l = w[136] * inv; w[136] = l;
      w[137] -= l * w[120];
      w[138] -= l * w[121];
      w[139] -= l * w[122];
      w[140] -= l * w[123];
      w[141] -= l * w[124];
      w[142] -= l * w[125];
    }
    { const R l = w[174] * inv; w[174] = l;
      w[175] -= l * w[120];
      w[176] -= l * w[121];
      w[177] -= l * w[122];
      w[178] -= l * w[123];
      w[179] -= l * w[124];
      w[180] -= l * w[125];
    }
    { const R l = w[191] * inv; w[191] = l;
      w[192] -= l * w[120];
      w[193] -= l * w[121];
      w[194] -= l * w[122];
      w[195] -= l * w[123];
      w[196] -= l * w[124];
      w[197] -= l * w[125];
    }
  }
  {  // pivot 23: state 12 (X_c), 4 rows x 5 cols
    const R pv = w[137];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::key(w[145]), P::key(w[155])), P::key(w[175])), P::key(w[192]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[137] = inv;
    { const R l = w[145] * inv; w[145] = l;
      w[146] -= l * w[138];
      w[147] -= l * w[139];
      w[148] -= l * w[140];
      w[149] -= l * w[141];
      w[150] -= l * w[142];
    }
    { const R l = w[155] * inv; w[155] = l;
      w[156] -= l * w[138];
      w[157] -= l * w[139];
      w[158] -= l * w[140];
      w[159] -= l * w[141];
      w[160] -= l * w[142];
    }
    { const R l = w[175] * inv; w[175] = l;
      w[176] -= l * w[138];
      w[177] -= l * w[139];
      w[178] -= l * w[140];
      w[179] -= l * w[141];
      w[180] -= l * w[142];
    }
    { const R l = w[192] * inv; w[192] = l;
      w[193] -= l * w[138];
      w[194] -= l * w[139];
      w[195] -= l * w[140];
      w[196] -= l * w[141];
      w[197] -= l * w[142];
    }
  }
  {  // pivot 24: state 3 (S_va), 4 rows x 4 cols
    const R pv = w[146];
    const typename P::K cm = P::kmax(P::kmax(P::kmax(P::key(w[156]), P::key(w[176])), P::key(w[193])), P::key(w[198]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[146] = inv;
    { const R l = w[156] * inv; w[156] = l;
      w[157] -= l * w[147];
      w[158] -= l * w[148];
      w[159] -= l * w[149];
      w[160] -= l * w[150];
    }
    { const R l = w[176] * inv; w[176] = l;
      w[177] -= l * w[147];
      w[178] -= l * w[148];
      w[179] -= l * w[149];
      w[180] -= l * w[150];
    }
    { const R l = w[193] * inv; w[193] = l;
      w[194] -= l * w[147];
      w[195] -= l * w[148];
      w[196] -= l * w[149];
      w[197] -= l * w[150];
    }
    { const R l = w[198] * inv; w[198] = l;
      w[199] -= l * w[147];
      w[200] -= l * w[148];
      w[201] -= l * w[149];
      w[202] -= l * w[150];
    }
  }
  {  // pivot 25: state 4 (S_bu), 3 rows x 3 cols
    const R pv = w[157];
    const typename P::K cm = P::kmax(P::kmax(P::key(w[177]), P::key(w[194])), P::key(w[199]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[157] = inv;
    { const R l = w[177] * inv; w[177] = l;
      w[178] -= l * w[158];
      w[179] -= l * w[159];
      w[180] -= l * w[160];
    }
    { const R l = w[194] * inv; w[194] = l;
      w[195] -= l * w[158];
      w[196] -= l * w[159];
      w[197] -= l * w[160];
    }
    { const R l = w[199] * inv; w[199] = l;
      w[200] -= l * w[158];
      w[201] -= l * w[159];
      w[202] -= l * w[160];
    }
  }
  {  // pivot 26: state 7 (S_h2), 2 rows x 2 cols
    const R pv = w[178];
    const typename P::K cm = P::kmax(P::key(w[195]), P::key(w[200]));
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[178] = inv;
    { const R l = w[195] * inv; w[195] = l;
      w[196] -= l * w[179];
      w[197] -= l * w[180];
    }
    { const R l = w[200] * inv; w[200] = l;
      w[201] -= l * w[179];
      w[202] -= l * w[180];
    }
  }
  {  // pivot 27: state 10 (S_IN), 1 rows x 1 cols
    const R pv = w[196];
    const typename P::K cm = P::key(w[201]);
    ok = ok && P::good(P::key(pv), cm);
    const R inv = rcp<R>(pv);
    w[196] = inv;
    { const R l = w[201] * inv; w[201] = l;
      w[202] -= l * w[197];
    }
  }
  {  // pivot 28: state 19 (X_c4), 0 rows x 0 cols
    const R pv = w[202];
    ok = ok && P::good(P::key(pv));
    const R inv = rcp<R>(pv);
    w[202] = inv;
  }
  return ok;
}

// Solve W x = b in place (b indexed by state).
template <class R, class W>
CHAD_HD void solve(W w, R* b) {
  R z0 = b[11];
  R z1 = b[23];
  R z2 = b[24];
  R z3 = b[25];
  R z4 = b[13];
  R z5 = b[14];
  R z6 = b[15];
  R z7 = b[8];
  R z8 = b[26];
  R z9 = b[28];
  R z10 = b[21];
  R z11 = b[22];
  R z12 = b[27];
  R z13 = b[9];
  R z14 = b[16];
  R z15 = b[0];
  R z16 = b[18];
  R z17 = b[2];
  R z18 = b[20];
  R z19 = b[17];
  R z20 = b[1];
  R z21 = b[6];
  R z22 = b[5];
  R z23 = b[12];
  R z24 = b[3];
  R z25 = b[4];
  R z26 = b[7];
  R z27 = b[10];
  R z28 = b[19];
  z9 -= w[23] * z8;
  z12 -= w[34] * z7;
  z12 -= w[35] * z8;
  z12 -= w[36] * z9;
  z12 -= w[37] * z10;
  z12 -= w[38] * z11;
  z13 -= w[44] * z4;
  z13 -= w[45] * z5;
  z13 -= w[46] * z6;
  z13 -= w[47] * z9;
  z13 -= w[48] * z10;
  z13 -= w[49] * z11;
  z13 -= w[50] * z12;
  z15 -= w[70] * z4;
  z15 -= w[71] * z6;
  z15 -= w[72] * z14;
  z17 -= w[80] * z6;
  z17 -= w[81] * z16;
  z20 -= w[93] * z5;
  z20 -= w[94] * z19;
  z21 -= w[98] * z10;
  z21 -= w[99] * z14;
  z21 -= w[100] * z15;
  z21 -= w[101] * z16;
  z21 -= w[102] * z17;
  z21 -= w[103] * z18;
  z21 -= w[104] * z19;
  z21 -= w[105] * z20;
  z22 -= w[114] * z14;
  z22 -= w[115] * z15;
  z22 -= w[116] * z18;
  z22 -= w[117] * z19;
  z22 -= w[118] * z20;
  z23 -= w[126] * z10;
  z23 -= w[127] * z11;
  z23 -= w[128] * z14;
  z23 -= w[129] * z15;
  z23 -= w[130] * z16;
  z23 -= w[131] * z17;
  z23 -= w[132] * z18;
  z23 -= w[133] * z19;
  z23 -= w[134] * z20;
  z23 -= w[135] * z21;
  z23 -= w[136] * z22;
  z24 -= w[143] * z19;
  z24 -= w[144] * z20;
  z24 -= w[145] * z23;
  z25 -= w[151] * z14;
  z25 -= w[152] * z15;
  z25 -= w[153] * z19;
  z25 -= w[154] * z20;
  z25 -= w[155] * z23;
  z25 -= w[156] * z24;
  z26 -= w[161] * z8;
  z26 -= w[162] * z9;
  z26 -= w[163] * z11;
  z26 -= w[164] * z12;
  z26 -= w[165] * z13;
  z26 -= w[166] * z14;
  z26 -= w[167] * z15;
  z26 -= w[168] * z16;
  z26 -= w[169] * z17;
  z26 -= w[170] * z18;
  z26 -= w[171] * z19;
  z26 -= w[172] * z20;
  z26 -= w[173] * z21;
  z26 -= w[174] * z22;
  z26 -= w[175] * z23;
  z26 -= w[176] * z24;
  z26 -= w[177] * z25;
  z27 -= w[181] * z10;
  z27 -= w[182] * z11;
  z27 -= w[183] * z14;
  z27 -= w[184] * z15;
  z27 -= w[185] * z16;
  z27 -= w[186] * z17;
  z27 -= w[187] * z18;
  z27 -= w[188] * z19;
  z27 -= w[189] * z20;
  z27 -= w[190] * z21;
  z27 -= w[191] * z22;
  z27 -= w[192] * z23;
  z27 -= w[193] * z24;
  z27 -= w[194] * z25;
  z27 -= w[195] * z26;
  z28 -= w[198] * z24;
  z28 -= w[199] * z25;
  z28 -= w[200] * z26;
  z28 -= w[201] * z27;
  z28 *= w[202];
  z27 -= w[197] * z28;
  z27 *= w[196];
  z26 -= w[179] * z27;
  z26 -= w[180] * z28;
  z26 *= w[178];
  z25 -= w[158] * z26;
  z25 -= w[159] * z27;
  z25 -= w[160] * z28;
  z25 *= w[157];
  z24 -= w[147] * z25;
  z24 -= w[148] * z26;
  z24 -= w[149] * z27;
  z24 -= w[150] * z28;
  z24 *= w[146];
  z23 -= w[138] * z24;
  z23 -= w[139] * z25;
  z23 -= w[140] * z26;
  z23 -= w[141] * z27;
  z23 -= w[142] * z28;
  z23 *= w[137];
  z22 -= w[120] * z23;
  z22 -= w[121] * z24;
  z22 -= w[122] * z25;
  z22 -= w[123] * z26;
  z22 -= w[124] * z27;
  z22 -= w[125] * z28;
  z22 *= w[119];
  z21 -= w[107] * z22;
  z21 -= w[108] * z23;
  z21 -= w[109] * z24;
  z21 -= w[110] * z25;
  z21 -= w[111] * z26;
  z21 -= w[112] * z27;
  z21 -= w[113] * z28;
  z21 *= w[106];
  z20 -= w[96] * z23;
  z20 -= w[97] * z27;
  z20 *= w[95];
  z19 -= w[91] * z20;
  z19 -= w[92] * z27;
  z19 *= w[90];
  z18 -= w[87] * z22;
  z18 -= w[88] * z26;
  z18 -= w[89] * z27;
  z18 *= w[86];
  z17 -= w[83] * z23;
  z17 -= w[84] * z26;
  z17 -= w[85] * z27;
  z17 *= w[82];
  z16 -= w[77] * z17;
  z16 -= w[78] * z26;
  z16 -= w[79] * z27;
  z16 *= w[76];
  z15 -= w[74] * z23;
  z15 -= w[75] * z27;
  z15 *= w[73];
  z14 -= w[68] * z15;
  z14 -= w[69] * z27;
  z14 *= w[67];
  z13 -= w[52] * z14;
  z13 -= w[53] * z15;
  z13 -= w[54] * z16;
  z13 -= w[55] * z17;
  z13 -= w[56] * z18;
  z13 -= w[57] * z19;
  z13 -= w[58] * z20;
  z13 -= w[59] * z21;
  z13 -= w[60] * z22;
  z13 -= w[61] * z23;
  z13 -= w[62] * z24;
  z13 -= w[63] * z25;
  z13 -= w[64] * z26;
  z13 -= w[65] * z27;
  z13 -= w[66] * z28;
  z13 *= w[51];
  z12 -= w[40] * z13;
  z12 -= w[41] * z21;
  z12 -= w[42] * z26;
  z12 -= w[43] * z27;
  z12 *= w[39];
  z11 -= w[32] * z26;
  z11 -= w[33] * z27;
  z11 *= w[31];
  z10 -= w[29] * z21;
  z10 -= w[30] * z27;
  z10 *= w[28];
  z9 -= w[25] * z12;
  z9 -= w[26] * z13;
  z9 -= w[27] * z26;
  z9 *= w[24];
  z8 -= w[20] * z9;
  z8 -= w[21] * z12;
  z8 -= w[22] * z26;
  z8 *= w[19];
  z7 -= w[13] * z10;
  z7 -= w[14] * z11;
  z7 -= w[15] * z12;
  z7 -= w[16] * z21;
  z7 -= w[17] * z26;
  z7 -= w[18] * z27;
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
  b[8] = z7;
  b[26] = z8;
  b[28] = z9;
  b[21] = z10;
  b[22] = z11;
  b[27] = z12;
  b[9] = z13;
  b[16] = z14;
  b[0] = z15;
  b[18] = z16;
  b[2] = z17;
  b[20] = z18;
  b[17] = z19;
  b[1] = z20;
  b[6] = z21;
  b[5] = z22;
  b[12] = z23;
  b[3] = z24;
  b[4] = z25;
  b[7] = z26;
  b[10] = z27;
  b[19] = z28;
}

constexpr int kFactorFlops = 640;
constexpr int kSolveFlops = 377;

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

}  // namespace sp
}  // namespace chad
