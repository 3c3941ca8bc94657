// GENERATED by gen_sparse.py from the library's own Jacobian pattern -- do not edit.
// Static-order (Markowitz) sparse LU of W = I - g J for the 29 ADM1 states.
// pattern nnz(J) = 279, slots with fill = 306
#pragma once
#include "adm1_device.cuh"

namespace chad {
namespace sp {

constexpr int kNNZ = 306;
constexpr int kNNZ_J = 279;
// elimination position -> state index
constexpr int kOrder[NS] = {11, 23, 24, 25, 13, 14, 15, 26, 27, 8, 28, 22, 21, 20, 2, 18, 0, 16, 19, 12, 7, 1, 3, 4, 5, 6, 9, 10, 17};

CHAD_HD constexpr int slot(int r, int c) {
  // row-major table over states, -1 = structurally zero
  const int t[NS * NS] = {
      108, -1, -1, 111, 112, 113, 114, -1, -1, 115, 116, -1, 110, 106, -1, 107, 109, -1, -1, -1, -1, -1, -1, -1, 104, 105, -1, -1, -1,
      -1, 182, -1, 183, 184, 185, 186, 181, -1, 187, 188, -1, 180, -1, 179, -1, -1, 189, -1, -1, -1, -1, -1, -1, 177, 178, -1, -1, -1,
      -1, -1, 82, 86, 87, 88, 89, 85, -1, 90, 91, -1, 84, -1, -1, 81, -1, -1, 83, -1, -1, -1, -1, -1, 79, 80, -1, -1, -1,
      -1, 194, -1, 195, 196, 197, 198, 193, -1, 199, 200, -1, -1, -1, -1, -1, -1, 201, -1, 192, -1, -1, -1, -1, 190, 191, -1, -1, -1,
      204, 209, -1, 210, 211, 212, 213, 208, -1, 214, 215, -1, 207, -1, -1, -1, 205, 216, -1, 206, -1, -1, -1, -1, 202, 203, -1, -1, -1,
      220, 225, -1, 226, 227, 228, 229, 224, -1, 230, 231, -1, 223, -1, -1, -1, 221, 232, -1, 222, 219, -1, -1, -1, 217, 218, -1, -1, -1,
      239, 244, 237, 245, 246, 247, 248, 243, -1, 249, 250, -1, 242, -1, -1, -1, 240, 251, 238, 241, 236, 235, -1, -1, 233, 234, -1, -1, -1,
      164, 169, 162, 170, 171, 172, 173, 168, 157, 174, 175, -1, 167, -1, -1, -1, 165, 176, 163, 166, 161, 160, 159, -1, 153, 154, 155, 156, 158,
      -1, -1, -1, 29, 30, 31, 32, 28, 24, 33, 34, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 27, 26, -1, 21, 22, -1, 23, 25,
      263, 268, 261, 269, 270, 271, 272, 267, -1, 273, 274, -1, 266, 254, 255, 256, 264, 275, 262, 265, 260, 259, 258, -1, 252, 253, -1, -1, 257,
      283, 288, 281, 289, 290, 291, 292, 287, -1, 293, 294, -1, 286, -1, -1, -1, 284, 295, 282, 285, 280, 279, 278, -1, 276, 277, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 0, 1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, 146, 147, 148, 149, 145, -1, 150, 151, -1, 144, -1, -1, -1, 142, 152, 141, 143, 140, 139, 138, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 7, 6, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 9, -1, 8, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 11, -1, -1, 10, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
      119, -1, -1, 122, 123, 124, 125, -1, -1, 126, 127, -1, 121, -1, -1, -1, 120, -1, -1, -1, -1, -1, -1, -1, 117, 118, -1, -1, -1,
      -1, 298, -1, 299, 300, 301, 302, -1, -1, 303, 304, -1, -1, -1, -1, -1, -1, 305, -1, -1, -1, -1, -1, -1, 296, 297, -1, -1, -1,
      -1, -1, 94, 98, 99, 100, 101, 97, -1, 102, 103, -1, 96, -1, -1, -1, -1, -1, 95, -1, -1, -1, -1, -1, 92, 93, -1, -1, -1,
      -1, -1, -1, 132, 133, 134, 135, 131, -1, 136, 137, -1, -1, -1, -1, -1, -1, -1, -1, 130, -1, -1, -1, -1, 128, 129, -1, -1, -1,
      -1, -1, -1, 73, 74, 75, 76, 72, -1, 77, 78, -1, -1, -1, -1, -1, -1, -1, -1, -1, 71, -1, -1, -1, 69, 70, -1, -1, -1,
      -1, -1, -1, 63, 64, 65, 66, -1, -1, 67, 68, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 62, -1, -1, 60, 61, -1, -1, -1,
      -1, -1, -1, 54, 55, 56, 57, 53, -1, 58, 59, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 52, -1, 50, 51, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 3, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 2, -1, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 4, -1, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 5, -1, -1, -1,
      -1, -1, -1, -1, -1, -1, -1, 15, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 12, 13, 14,
      -1, -1, -1, -1, -1, -1, -1, 20, 18, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 16, 17, 19,
      -1, -1, -1, 44, 45, 46, 47, 43, 39, 48, 49, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 42, 41, -1, 35, 36, 37, 38, 40
  };
  return t[r * NS + c];
}

struct Idx {
  static CHAD_HD constexpr int at(int r, int c) { return slot(r, c); }
  static constexpr int size = kNNZ;
};

// diagonal slots in elimination order
constexpr int kDiag[NS] = {0, 2, 4, 5, 6, 8, 10, 12, 17, 24, 40, 52, 62, 71, 82, 95, 108, 120, 130, 144, 168, 182, 195, 211, 228, 248, 273, 294, 305};

// W = I - g J in place over the slots (fill slots hold zero in J)
template <class R>
CHAD_HD void form_w(R* w, R g) {
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
  w[17] += R(1);
  w[24] += R(1);
  w[40] += R(1);
  w[52] += R(1);
  w[62] += R(1);
  w[71] += R(1);
  w[82] += R(1);
  w[95] += R(1);
  w[108] += R(1);
  w[120] += R(1);
  w[130] += R(1);
  w[144] += R(1);
  w[168] += R(1);
  w[182] += R(1);
  w[195] += R(1);
  w[211] += R(1);
  w[228] += R(1);
  w[248] += R(1);
  w[273] += R(1);
  w[294] += R(1);
  w[305] += R(1);
}

// In-place LU; returns false if a pivot fails the threshold test.
template <class R>
CHAD_HD bool factor(R* w, R* dinv, R tau) {
  bool ok = true;
  {  // pivot 0: state 11 (S_I), 0 rows x 1 cols
    const R pv = w[0];
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[0] = inv;
  }
  {  // pivot 1: state 23 (X_I), 0 rows x 1 cols
    const R pv = w[2];
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[1] = inv;
  }
  {  // pivot 2: state 24 (S_cat), 19 rows x 0 cols
    const R pv = w[4];
    const R cm = fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fabs(w[21]), fabs(w[35])), fabs(w[50])), fabs(w[60])), fabs(w[69])), fabs(w[79])), fabs(w[92])), fabs(w[104])), fabs(w[117])), fabs(w[128])), fabs(w[153])), fabs(w[177])), fabs(w[190])), fabs(w[202])), fabs(w[217])), fabs(w[233])), fabs(w[252])), fabs(w[276])), fabs(w[296]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[2] = inv;
    { const R l = w[21] * inv; w[21] = l;
    }
    { const R l = w[35] * inv; w[35] = l;
    }
    { const R l = w[50] * inv; w[50] = l;
    }
    { const R l = w[60] * inv; w[60] = l;
    }
    { const R l = w[69] * inv; w[69] = l;
    }
    { const R l = w[79] * inv; w[79] = l;
    }
    { const R l = w[92] * inv; w[92] = l;
    }
    { const R l = w[104] * inv; w[104] = l;
    }
    { const R l = w[117] * inv; w[117] = l;
    }
    { const R l = w[128] * inv; w[128] = l;
    }
    { const R l = w[153] * inv; w[153] = l;
    }
    { const R l = w[177] * inv; w[177] = l;
    }
    { const R l = w[190] * inv; w[190] = l;
    }
    { const R l = w[202] * inv; w[202] = l;
    }
    { const R l = w[217] * inv; w[217] = l;
    }
    { const R l = w[233] * inv; w[233] = l;
    }
    { const R l = w[252] * inv; w[252] = l;
    }
    { const R l = w[276] * inv; w[276] = l;
    }
    { const R l = w[296] * inv; w[296] = l;
    }
  }
  {  // pivot 3: state 25 (S_an), 19 rows x 0 cols
    const R pv = w[5];
    const R cm = fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fmax(fabs(w[22]), fabs(w[36])), fabs(w[51])), fabs(w[61])), fabs(w[70])), fabs(w[80])), fabs(w[93])), fabs(w[105])), fabs(w[118])), fabs(w[129])), fabs(w[154])), fabs(w[178])), fabs(w[191])), fabs(w[203])), fabs(w[218])), fabs(w[234])), fabs(w[253])), fabs(w[277])), fabs(w[297]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[3] = inv;
    { const R l = w[22] * inv; w[22] = l;
    }
    { const R l = w[36] * inv; w[36] = l;
    }
    { const R l = w[51] * inv; w[51] = l;
    }
    { const R l = w[61] * inv; w[61] = l;
    }
    { const R l = w[70] * inv; w[70] = l;
    }
    { const R l = w[80] * inv; w[80] = l;
    }
    { const R l = w[93] * inv; w[93] = l;
    }
    { const R l = w[105] * inv; w[105] = l;
    }
    { const R l = w[118] * inv; w[118] = l;
    }
    { const R l = w[129] * inv; w[129] = l;
    }
    { const R l = w[154] * inv; w[154] = l;
    }
    { const R l = w[178] * inv; w[178] = l;
    }
    { const R l = w[191] * inv; w[191] = l;
    }
    { const R l = w[203] * inv; w[203] = l;
    }
    { const R l = w[218] * inv; w[218] = l;
    }
    { const R l = w[234] * inv; w[234] = l;
    }
    { const R l = w[253] * inv; w[253] = l;
    }
    { const R l = w[277] * inv; w[277] = l;
    }
    { const R l = w[297] * inv; w[297] = l;
    }
  }
  {  // pivot 4: state 13 (X_ch), 2 rows x 1 cols
    const R pv = w[6];
    const R cm = fmax(fabs(w[106]), fabs(w[254]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[4] = inv;
    { const R l = w[106] * inv; w[106] = l;
      w[110] -= l * w[7];
    }
    { const R l = w[254] * inv; w[254] = l;
      w[266] -= l * w[7];
    }
  }
  {  // pivot 5: state 14 (X_pr), 2 rows x 1 cols
    const R pv = w[8];
    const R cm = fmax(fabs(w[179]), fabs(w[255]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[5] = inv;
    { const R l = w[179] * inv; w[179] = l;
      w[180] -= l * w[9];
    }
    { const R l = w[255] * inv; w[255] = l;
      w[266] -= l * w[9];
    }
  }
  {  // pivot 6: state 15 (X_li), 3 rows x 1 cols
    const R pv = w[10];
    const R cm = fmax(fmax(fabs(w[81]), fabs(w[107])), fabs(w[256]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[6] = inv;
    { const R l = w[81] * inv; w[81] = l;
      w[84] -= l * w[11];
    }
    { const R l = w[107] * inv; w[107] = l;
      w[110] -= l * w[11];
    }
    { const R l = w[256] * inv; w[256] = l;
      w[266] -= l * w[11];
    }
  }
  {  // pivot 7: state 26 (S_gas_h2), 3 rows x 3 cols
    const R pv = w[12];
    const R cm = fmax(fmax(fabs(w[16]), fabs(w[37])), fabs(w[155]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[7] = inv;
    { const R l = w[16] * inv; w[16] = l;
      w[17] -= l * w[13];
      w[19] -= l * w[14];
      w[20] -= l * w[15];
    }
    { const R l = w[37] * inv; w[37] = l;
      w[38] -= l * w[13];
      w[40] -= l * w[14];
      w[43] -= l * w[15];
    }
    { const R l = w[155] * inv; w[155] = l;
      w[156] -= l * w[13];
      w[158] -= l * w[14];
      w[168] -= l * w[15];
    }
  }
  {  // pivot 8: state 27 (S_gas_ch4), 3 rows x 3 cols
    const R pv = w[17];
    const R cm = fmax(fmax(fabs(w[23]), fabs(w[38])), fabs(w[156]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[8] = inv;
    { const R l = w[23] * inv; w[23] = l;
      w[24] -= l * w[18];
      w[25] -= l * w[19];
      w[28] -= l * w[20];
    }
    { const R l = w[38] * inv; w[38] = l;
      w[39] -= l * w[18];
      w[40] -= l * w[19];
      w[43] -= l * w[20];
    }
    { const R l = w[156] * inv; w[156] = l;
      w[157] -= l * w[18];
      w[158] -= l * w[19];
      w[168] -= l * w[20];
    }
  }
  {  // pivot 9: state 8 (S_ch4), 2 rows x 10 cols
    const R pv = w[24];
    const R cm = fmax(fabs(w[39]), fabs(w[157]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[9] = inv;
    { const R l = w[39] * inv; w[39] = l;
      w[40] -= l * w[25];
      w[41] -= l * w[26];
      w[42] -= l * w[27];
      w[43] -= l * w[28];
      w[44] -= l * w[29];
      w[45] -= l * w[30];
      w[46] -= l * w[31];
      w[47] -= l * w[32];
      w[48] -= l * w[33];
      w[49] -= l * w[34];
    }
    { const R l = w[157] * inv; w[157] = l;
      w[158] -= l * w[25];
      w[159] -= l * w[26];
      w[160] -= l * w[27];
      w[168] -= l * w[28];
      w[170] -= l * w[29];
      w[171] -= l * w[30];
      w[172] -= l * w[31];
      w[173] -= l * w[32];
      w[174] -= l * w[33];
      w[175] -= l * w[34];
    }
  }
  {  // pivot 10: state 28 (S_gas_co2), 2 rows x 9 cols
    const R pv = w[40];
    const R cm = fmax(fabs(w[158]), fabs(w[257]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[10] = inv;
    { const R l = w[158] * inv; w[158] = l;
      w[159] -= l * w[41];
      w[160] -= l * w[42];
      w[168] -= l * w[43];
      w[170] -= l * w[44];
      w[171] -= l * w[45];
      w[172] -= l * w[46];
      w[173] -= l * w[47];
      w[174] -= l * w[48];
      w[175] -= l * w[49];
    }
    { const R l = w[257] * inv; w[257] = l;
      w[258] -= l * w[41];
      w[259] -= l * w[42];
      w[267] -= l * w[43];
      w[269] -= l * w[44];
      w[270] -= l * w[45];
      w[271] -= l * w[46];
      w[272] -= l * w[47];
      w[273] -= l * w[48];
      w[274] -= l * w[49];
    }
  }
  {  // pivot 11: state 22 (X_h2), 4 rows x 7 cols
    const R pv = w[52];
    const R cm = fmax(fmax(fmax(fabs(w[138]), fabs(w[159])), fabs(w[258])), fabs(w[278]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[11] = inv;
    { const R l = w[138] * inv; w[138] = l;
      w[145] -= l * w[53];
      w[146] -= l * w[54];
      w[147] -= l * w[55];
      w[148] -= l * w[56];
      w[149] -= l * w[57];
      w[150] -= l * w[58];
      w[151] -= l * w[59];
    }
    { const R l = w[159] * inv; w[159] = l;
      w[168] -= l * w[53];
      w[170] -= l * w[54];
      w[171] -= l * w[55];
      w[172] -= l * w[56];
      w[173] -= l * w[57];
      w[174] -= l * w[58];
      w[175] -= l * w[59];
    }
    { const R l = w[258] * inv; w[258] = l;
      w[267] -= l * w[53];
      w[269] -= l * w[54];
      w[270] -= l * w[55];
      w[271] -= l * w[56];
      w[272] -= l * w[57];
      w[273] -= l * w[58];
      w[274] -= l * w[59];
    }
    { const R l = w[278] * inv; w[278] = l;
      w[287] -= l * w[53];
      w[289] -= l * w[54];
      w[290] -= l * w[55];
      w[291] -= l * w[56];
      w[292] -= l * w[57];
      w[293] -= l * w[58];
      w[294] -= l * w[59];
    }
  }
  {  // pivot 12: state 21 (X_ac), 5 rows x 6 cols
    const R pv = w[62];
    const R cm = fmax(fmax(fmax(fmax(fabs(w[139]), fabs(w[160])), fabs(w[235])), fabs(w[259])), fabs(w[279]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[12] = inv;
    { const R l = w[139] * inv; w[139] = l;
      w[146] -= l * w[63];
      w[147] -= l * w[64];
      w[148] -= l * w[65];
      w[149] -= l * w[66];
      w[150] -= l * w[67];
      w[151] -= l * w[68];
    }
    { const R l = w[160] * inv; w[160] = l;
      w[170] -= l * w[63];
      w[171] -= l * w[64];
      w[172] -= l * w[65];
      w[173] -= l * w[66];
      w[174] -= l * w[67];
      w[175] -= l * w[68];
    }
    { const R l = w[235] * inv; w[235] = l;
      w[245] -= l * w[63];
      w[246] -= l * w[64];
      w[247] -= l * w[65];
      w[248] -= l * w[66];
      w[249] -= l * w[67];
      w[250] -= l * w[68];
    }
    { const R l = w[259] * inv; w[259] = l;
      w[269] -= l * w[63];
      w[270] -= l * w[64];
      w[271] -= l * w[65];
      w[272] -= l * w[66];
      w[273] -= l * w[67];
      w[274] -= l * w[68];
    }
    { const R l = w[279] * inv; w[279] = l;
      w[289] -= l * w[63];
      w[290] -= l * w[64];
      w[291] -= l * w[65];
      w[292] -= l * w[66];
      w[293] -= l * w[67];
      w[294] -= l * w[68];
    }
  }
  {  // pivot 13: state 20 (X_pro), 6 rows x 7 cols
    const R pv = w[71];
    const R cm = fmax(fmax(fmax(fmax(fmax(fabs(w[140]), fabs(w[161])), fabs(w[219])), fabs(w[236])), fabs(w[260])), fabs(w[280]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[13] = inv;
    { const R l = w[140] * inv; w[140] = l;
      w[145] -= l * w[72];
      w[146] -= l * w[73];
      w[147] -= l * w[74];
      w[148] -= l * w[75];
      w[149] -= l * w[76];
      w[150] -= l * w[77];
      w[151] -= l * w[78];
    }
    { const R l = w[161] * inv; w[161] = l;
      w[168] -= l * w[72];
      w[170] -= l * w[73];
      w[171] -= l * w[74];
      w[172] -= l * w[75];
      w[173] -= l * w[76];
      w[174] -= l * w[77];
      w[175] -= l * w[78];
    }
    { const R l = w[219] * inv; w[219] = l;
      w[224] -= l * w[72];
      w[226] -= l * w[73];
      w[227] -= l * w[74];
      w[228] -= l * w[75];
      w[229] -= l * w[76];
      w[230] -= l * w[77];
      w[231] -= l * w[78];
    }
    { const R l = w[236] * inv; w[236] = l;
      w[243] -= l * w[72];
      w[245] -= l * w[73];
      w[246] -= l * w[74];
      w[247] -= l * w[75];
      w[248] -= l * w[76];
      w[249] -= l * w[77];
      w[250] -= l * w[78];
    }
    { const R l = w[260] * inv; w[260] = l;
      w[267] -= l * w[72];
      w[269] -= l * w[73];
      w[270] -= l * w[74];
      w[271] -= l * w[75];
      w[272] -= l * w[76];
      w[273] -= l * w[77];
      w[274] -= l * w[78];
    }
    { const R l = w[280] * inv; w[280] = l;
      w[287] -= l * w[72];
      w[289] -= l * w[73];
      w[290] -= l * w[74];
      w[291] -= l * w[75];
      w[292] -= l * w[76];
      w[293] -= l * w[77];
      w[294] -= l * w[78];
    }
  }
  {  // pivot 14: state 2 (S_fa), 5 rows x 9 cols
    const R pv = w[82];
    const R cm = fmax(fmax(fmax(fmax(fabs(w[94]), fabs(w[162])), fabs(w[237])), fabs(w[261])), fabs(w[281]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[14] = inv;
    { const R l = w[94] * inv; w[94] = l;
      w[95] -= l * w[83];
      w[96] -= l * w[84];
      w[97] -= l * w[85];
      w[98] -= l * w[86];
      w[99] -= l * w[87];
      w[100] -= l * w[88];
      w[101] -= l * w[89];
      w[102] -= l * w[90];
      w[103] -= l * w[91];
    }
    { const R l = w[162] * inv; w[162] = l;
      w[163] -= l * w[83];
      w[167] -= l * w[84];
      w[168] -= l * w[85];
      w[170] -= l * w[86];
      w[171] -= l * w[87];
      w[172] -= l * w[88];
      w[173] -= l * w[89];
      w[174] -= l * w[90];
      w[175] -= l * w[91];
    }
    { const R l = w[237] * inv; w[237] = l;
      w[238] -= l * w[83];
      w[242] -= l * w[84];
      w[243] -= l * w[85];
      w[245] -= l * w[86];
      w[246] -= l * w[87];
      w[247] -= l * w[88];
      w[248] -= l * w[89];
      w[249] -= l * w[90];
      w[250] -= l * w[91];
    }
    { const R l = w[261] * inv; w[261] = l;
      w[262] -= l * w[83];
      w[266] -= l * w[84];
      w[267] -= l * w[85];
      w[269] -= l * w[86];
      w[270] -= l * w[87];
      w[271] -= l * w[88];
      w[272] -= l * w[89];
      w[273] -= l * w[90];
      w[274] -= l * w[91];
    }
    { const R l = w[281] * inv; w[281] = l;
      w[282] -= l * w[83];
      w[286] -= l * w[84];
      w[287] -= l * w[85];
      w[289] -= l * w[86];
      w[290] -= l * w[87];
      w[291] -= l * w[88];
      w[292] -= l * w[89];
      w[293] -= l * w[90];
      w[294] -= l * w[91];
    }
  }
  {  // pivot 15: state 18 (X_fa), 5 rows x 8 cols
    const R pv = w[95];
    const R cm = fmax(fmax(fmax(fmax(fabs(w[141]), fabs(w[163])), fabs(w[238])), fabs(w[262])), fabs(w[282]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[15] = inv;
    { const R l = w[141] * inv; w[141] = l;
      w[144] -= l * w[96];
      w[145] -= l * w[97];
      w[146] -= l * w[98];
      w[147] -= l * w[99];
      w[148] -= l * w[100];
      w[149] -= l * w[101];
      w[150] -= l * w[102];
      w[151] -= l * w[103];
    }
    { const R l = w[163] * inv; w[163] = l;
      w[167] -= l * w[96];
      w[168] -= l * w[97];
      w[170] -= l * w[98];
      w[171] -= l * w[99];
      w[172] -= l * w[100];
      w[173] -= l * w[101];
      w[174] -= l * w[102];
      w[175] -= l * w[103];
    }
    { const R l = w[238] * inv; w[238] = l;
      w[242] -= l * w[96];
      w[243] -= l * w[97];
      w[245] -= l * w[98];
      w[246] -= l * w[99];
      w[247] -= l * w[100];
      w[248] -= l * w[101];
      w[249] -= l * w[102];
      w[250] -= l * w[103];
    }
    { const R l = w[262] * inv; w[262] = l;
      w[266] -= l * w[96];
      w[267] -= l * w[97];
      w[269] -= l * w[98];
      w[270] -= l * w[99];
      w[271] -= l * w[100];
      w[272] -= l * w[101];
      w[273] -= l * w[102];
      w[274] -= l * w[103];
    }
    { const R l = w[282] * inv; w[282] = l;
      w[286] -= l * w[96];
      w[287] -= l * w[97];
      w[289] -= l * w[98];
      w[290] -= l * w[99];
      w[291] -= l * w[100];
      w[292] -= l * w[101];
      w[293] -= l * w[102];
      w[294] -= l * w[103];
    }
  }
  {  // pivot 16: state 0 (S_su), 7 rows x 8 cols
    const R pv = w[108];
    const R cm = fmax(fmax(fmax(fmax(fmax(fmax(fabs(w[119]), fabs(w[164])), fabs(w[204])), fabs(w[220])), fabs(w[239])), fabs(w[263])), fabs(w[283]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[16] = inv;
    { const R l = w[119] * inv; w[119] = l;
      w[120] -= l * w[109];
      w[121] -= l * w[110];
      w[122] -= l * w[111];
      w[123] -= l * w[112];
      w[124] -= l * w[113];
      w[125] -= l * w[114];
      w[126] -= l * w[115];
      w[127] -= l * w[116];
    }
    { const R l = w[164] * inv; w[164] = l;
      w[165] -= l * w[109];
      w[167] -= l * w[110];
      w[170] -= l * w[111];
      w[171] -= l * w[112];
      w[172] -= l * w[113];
      w[173] -= l * w[114];
      w[174] -= l * w[115];
      w[175] -= l * w[116];
    }
    { const R l = w[204] * inv; w[204] = l;
      w[205] -= l * w[109];
      w[207] -= l * w[110];
      w[210] -= l * w[111];
      w[211] -= l * w[112];
      w[212] -= l * w[113];
      w[213] -= l * w[114];
      w[214] -= l * w[115];
      w[215] -= l * w[116];
    }
    { const R l = w[220] * inv; w[220] = l;
      w[221] -= l * w[109];
      w[223] -= l * w[110];
      w[226] -= l * w[111];
      w[227] -= l * w[112];
      w[228] -= l * w[113];
      w[229] -= l * w[114];
      w[230] -= l * w[115];
      w[231] -= l * w[116];
    }
    { const R l = w[239] * inv; w[239] = l;
      w[240] -= l * w[109];
      w[242] -= l * w[110];
      w[245] -= l * w[111];
      w[246] -= l * w[112];
      w[247] -= l * w[113];
      w[248] -= l * w[114];
      w[249] -= l * w[115];
      w[250] -= l * w[116];
    }
    { const R l = w[263] * inv; w[263] = l;
      w[264] -= l * w[109];
      w[266] -= l * w[110];
      w[269] -= l * w[111];
      w[270] -= l * w[112];
      w[271] -= l * w[113];
      w[272] -= l * w[114];
      w[273] -= l * w[115];
      w[274] -= l * w[116];
    }
    { const R l = w[283] * inv; w[283] = l;
      w[284] -= l * w[109];
      w[286] -= l * w[110];
      w[289] -= l * w[111];
      w[290] -= l * w[112];
      w[291] -= l * w[113];
      w[292] -= l * w[114];
      w[293] -= l * w[115];
      w[294] -= l * w[116];
    }
  }
  {  // pivot 17: state 16 (X_su), 7 rows x 7 cols
    const R pv = w[120];
    const R cm = fmax(fmax(fmax(fmax(fmax(fmax(fabs(w[142]), fabs(w[165])), fabs(w[205])), fabs(w[221])), fabs(w[240])), fabs(w[264])), fabs(w[284]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[17] = inv;
    { const R l = w[142] * inv; w[142] = l;
      w[144] -= l * w[121];
      w[146] -= l * w[122];
      w[147] -= l * w[123];
      w[148] -= l * w[124];
      w[149] -= l * w[125];
      w[150] -= l * w[126];
      w[151] -= l * w[127];
    }
    { const R l = w[165] * inv; w[165] = l;
      w[167] -= l * w[121];
      w[170] -= l * w[122];
      w[171] -= l * w[123];
      w[172] -= l * w[124];
      w[173] -= l * w[125];
      w[174] -= l * w[126];
      w[175] -= l * w[127];
    }
    { const R l = w[205] * inv; w[205] = l;
      w[207] -= l * w[121];
      w[210] -= l * w[122];
      w[211] -= l * w[123];
      w[212] -= l * w[124];
      w[213] -= l * w[125];
      w[214] -= l * w[126];
      w[215] -= l * w[127];
    }
    { const R l = w[221] * inv; w[221] = l;
      w[223] -= l * w[121];
      w[226] -= l * w[122];
      w[227] -= l * w[123];
      w[228] -= l * w[124];
      w[229] -= l * w[125];
      w[230] -= l * w[126];
      w[231] -= l * w[127];
    }
    { const R l = w[240] * inv; w[240] = l;
      w[242] -= l * w[121];
      w[245] -= l * w[122];
      w[246] -= l * w[123];
      w[247] -= l * w[124];
      w[248] -= l * w[125];
      w[249] -= l * w[126];
      w[250] -= l * w[127];
    }
    { const R l = w[264] * inv; w[264] = l;
      w[266] -= l * w[121];
      w[269] -= l * w[122];
      w[270] -= l * w[123];
      w[271] -= l * w[124];
      w[272] -= l * w[125];
      w[273] -= l * w[126];
      w[274] -= l * w[127];
    }
    { const R l = w[284] * inv; w[284] = l;
      w[286] -= l * w[121];
      w[289] -= l * w[122];
      w[290] -= l * w[123];
      w[291] -= l * w[124];
      w[292] -= l * w[125];
      w[293] -= l * w[126];
      w[294] -= l * w[127];
    }
  }
  {  // pivot 18: state 19 (X_c4), 8 rows x 7 cols
    const R pv = w[130];
    const R cm = fmax(fmax(fmax(fmax(fmax(fmax(fmax(fabs(w[143]), fabs(w[166])), fabs(w[192])), fabs(w[206])), fabs(w[222])), fabs(w[241])), fabs(w[265])), fabs(w[285]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[18] = inv;
    { const R l = w[143] * inv; w[143] = l;
      w[145] -= l * w[131];
      w[146] -= l * w[132];
      w[147] -= l * w[133];
      w[148] -= l * w[134];
      w[149] -= l * w[135];
      w[150] -= l * w[136];
      w[151] -= l * w[137];
    }
    { const R l = w[166] * inv; w[166] = l;
      w[168] -= l * w[131];
      w[170] -= l * w[132];
      w[171] -= l * w[133];
      w[172] -= l * w[134];
      w[173] -= l * w[135];
      w[174] -= l * w[136];
      w[175] -= l * w[137];
    }
    { const R l = w[192] * inv; w[192] = l;
      w[193] -= l * w[131];
      w[195] -= l * w[132];
      w[196] -= l * w[133];
      w[197] -= l * w[134];
      w[198] -= l * w[135];
      w[199] -= l * w[136];
      w[200] -= l * w[137];
    }
    { const R l = w[206] * inv; w[206] = l;
      w[208] -= l * w[131];
      w[210] -= l * w[132];
      w[211] -= l * w[133];
      w[212] -= l * w[134];
      w[213] -= l * w[135];
      w[214] -= l * w[136];
      w[215] -= l * w[137];
    }
    { const R l = w[222] * inv; w[222] = l;
      w[224] -= l * w[131];
      w[226] -= l * w[132];
      w[227] -= l * w[133];
      w[228] -= l * w[134];
      w[229] -= l * w[135];
      w[230] -= l * w[136];
      w[231] -= l * w[137];
    }
    { const R l = w[241] * inv; w[241] = l;
      w[243] -= l * w[131];
      w[245] -= l * w[132];
      w[246] -= l * w[133];
      w[247] -= l * w[134];
      w[248] -= l * w[135];
      w[249] -= l * w[136];
      w[250] -= l * w[137];
    }
    { const R l = w[265] * inv; w[265] = l;
      w[267] -= l * w[131];
      w[269] -= l * w[132];
      w[270] -= l * w[133];
      w[271] -= l * w[134];
      w[272] -= l * w[135];
      w[273] -= l * w[136];
      w[274] -= l * w[137];
    }
    { const R l = w[285] * inv; w[285] = l;
      w[287] -= l * w[131];
      w[289] -= l * w[132];
      w[290] -= l * w[133];
      w[291] -= l * w[134];
      w[292] -= l * w[135];
      w[293] -= l * w[136];
      w[294] -= l * w[137];
    }
  }
  {  // pivot 19: state 12 (X_c), 7 rows x 8 cols
    const R pv = w[144];
    const R cm = fmax(fmax(fmax(fmax(fmax(fmax(fabs(w[167]), fabs(w[180])), fabs(w[207])), fabs(w[223])), fabs(w[242])), fabs(w[266])), fabs(w[286]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[19] = inv;
    { const R l = w[167] * inv; w[167] = l;
      w[168] -= l * w[145];
      w[170] -= l * w[146];
      w[171] -= l * w[147];
      w[172] -= l * w[148];
      w[173] -= l * w[149];
      w[174] -= l * w[150];
      w[175] -= l * w[151];
      w[176] -= l * w[152];
    }
    { const R l = w[180] * inv; w[180] = l;
      w[181] -= l * w[145];
      w[183] -= l * w[146];
      w[184] -= l * w[147];
      w[185] -= l * w[148];
      w[186] -= l * w[149];
      w[187] -= l * w[150];
      w[188] -= l * w[151];
      w[189] -= l * w[152];
    }
    { const R l = w[207] * inv; w[207] = l;
      w[208] -= l * w[145];
      w[210] -= l * w[146];
      w[211] -= l * w[147];
      w[212] -= l * w[148];
      w[213] -= l * w[149];
      w[214] -= l * w[150];
      w[215] -= l * w[151];
      w[216] -= l * w[152];
    }
    { const R l = w[223] * inv; w[223] = l;
      w[224] -= l * w[145];
      w[226] -= l * w[146];
      w[227] -= l * w[147];
      w[228] -= l * w[148];
      w[229] -= l * w[149];
      w[230] -= l * w[150];
      w[231] -= l * w[151];
      w[232] -= l * w[152];
    }
    { const R l = w[242] * inv; w[242] = l;
      w[243] -= l * w[145];
      w[245] -= l * w[146];
      w[246] -= l * w[147];
      w[247] -= l * w[148];
      w[248] -= l * w[149];
      w[249] -= l * w[150];
      w[250] -= l * w[151];
      w[251] -= l * w[152];
    }
    { const R l = w[266] * inv; w[266] = l;
      w[267] -= l * w[145];
      w[269] -= l * w[146];
      w[270] -= l * w[147];
      w[271] -= l * w[148];
      w[272] -= l * w[149];
      w[273] -= l * w[150];
      w[274] -= l * w[151];
      w[275] -= l * w[152];
    }
    { const R l = w[286] * inv; w[286] = l;
      w[287] -= l * w[145];
      w[289] -= l * w[146];
      w[290] -= l * w[147];
      w[291] -= l * w[148];
      w[292] -= l * w[149];
      w[293] -= l * w[150];
      w[294] -= l * w[151];
      w[295] -= l * w[152];
    }
  }
  {  // pivot 20: state 7 (S_h2), 7 rows x 8 cols
    const R pv = w[168];
    const R cm = fmax(fmax(fmax(fmax(fmax(fmax(fabs(w[181]), fabs(w[193])), fabs(w[208])), fabs(w[224])), fabs(w[243])), fabs(w[267])), fabs(w[287]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[20] = inv;
    { const R l = w[181] * inv; w[181] = l;
      w[182] -= l * w[169];
      w[183] -= l * w[170];
      w[184] -= l * w[171];
      w[185] -= l * w[172];
      w[186] -= l * w[173];
      w[187] -= l * w[174];
      w[188] -= l * w[175];
      w[189] -= l * w[176];
    }
    { const R l = w[193] * inv; w[193] = l;
      w[194] -= l * w[169];
      w[195] -= l * w[170];
      w[196] -= l * w[171];
      w[197] -= l * w[172];
      w[198] -= l * w[173];
      w[199] -= l * w[174];
      w[200] -= l * w[175];
      w[201] -= l * w[176];
    }
    { const R l = w[208] * inv; w[208] = l;
      w[209] -= l * w[169];
      w[210] -= l * w[170];
      w[211] -= l * w[171];
      w[212] -= l * w[172];
      w[213] -= l * w[173];
      w[214] -= l * w[174];
      w[215] -= l * w[175];
      w[216] -= l * w[176];
    }
    { const R l = w[224] * inv; w[224] = l;
      w[225] -= l * w[169];
      w[226] -= l * w[170];
      w[227] -= l * w[171];
      w[228] -= l * w[172];
      w[229] -= l * w[173];
      w[230] -= l * w[174];
      w[231] -= l * w[175];
      w[232] -= l * w[176];
    }
    { const R l = w[243] * inv; w[243] = l;
      w[244] -= l * w[169];
      w[245] -= l * w[170];
      w[246] -= l * w[171];
      w[247] -= l * w[172];
      w[248] -= l * w[173];
      w[249] -= l * w[174];
      w[250] -= l * w[175];
      w[251] -= l * w[176];
    }
    { const R l = w[267] * inv; w[267] = l;
      w[268] -= l * w[169];
      w[269] -= l * w[170];
      w[270] -= l * w[171];
      w[271] -= l * w[172];
      w[272] -= l * w[173];
      w[273] -= l * w[174];
      w[274] -= l * w[175];
      w[275] -= l * w[176];
    }
    { const R l = w[287] * inv; w[287] = l;
      w[288] -= l * w[169];
      w[289] -= l * w[170];
      w[290] -= l * w[171];
      w[291] -= l * w[172];
      w[292] -= l * w[173];
      w[293] -= l * w[174];
      w[294] -= l * w[175];
      w[295] -= l * w[176];
    }
  }
  {  // pivot 21: state 1 (S_aa), 7 rows x 7 cols
    const R pv = w[182];
    const R cm = fmax(fmax(fmax(fmax(fmax(fmax(fabs(w[194]), fabs(w[209])), fabs(w[225])), fabs(w[244])), fabs(w[268])), fabs(w[288])), fabs(w[298]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[21] = inv;
    { const R l = w[194] * inv; w[194] = l;
      w[195] -= l * w[183];
      w[196] -= l * w[184];
      w[197] -= l * w[185];
      w[198] -= l * w[186];
      w[199] -= l * w[187];
      w[200] -= l * w[188];
      w[201] -= l * w[189];
    }
    { const R l = w[209] * inv; w[209] = l;
      w[210] -= l * w[183];
      w[211] -= l * w[184];
      w[212] -= l * w[185];
      w[213] -= l * w[186];
      w[214] -= l * w[187];
      w[215] -= l * w[188];
      w[216] -= l * w[189];
    }
    { const R l = w[225] * inv; w[225] = l;
      w[226] -= l * w[183];
      w[227] -= l * w[184];
      w[228] -= l * w[185];
      w[229] -= l * w[186];
      w[230] -= l * w[187];
      w[231] -= l * w[188];
      w[232] -= l * w[189];
    }
    { const R l = w[244] * inv; w[244] = l;
      w[245] -= l * w[183];
      w[246] -= l * w[184];
      w[247] -= l * w[185];
      w[248] -= l * w[186];
      w[249] -= l * w[187];
      w[250] -= l * w[188];
      w[251] -= l * w[189];
    }
    { const R l = w[268] * inv; w[268] = l;
      w[269] -= l * w[183];
      w[270] -= l * w[184];
      w[271] -= l * w[185];
      w[272] -= l * w[186];
      w[273] -= l * w[187];
      w[274] -= l * w[188];
      w[275] -= l * w[189];
    }
    { const R l = w[288] * inv; w[288] = l;
      w[289] -= l * w[183];
      w[290] -= l * w[184];
      w[291] -= l * w[185];
      w[292] -= l * w[186];
      w[293] -= l * w[187];
      w[294] -= l * w[188];
      w[295] -= l * w[189];
    }
    { const R l = w[298] * inv; w[298] = l;
      w[299] -= l * w[183];
      w[300] -= l * w[184];
      w[301] -= l * w[185];
      w[302] -= l * w[186];
      w[303] -= l * w[187];
      w[304] -= l * w[188];
      w[305] -= l * w[189];
    }
  }
  {  // pivot 22: state 3 (S_va), 6 rows x 6 cols
    const R pv = w[195];
    const R cm = fmax(fmax(fmax(fmax(fmax(fabs(w[210]), fabs(w[226])), fabs(w[245])), fabs(w[269])), fabs(w[289])), fabs(w[299]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[22] = inv;
    { const R l = w[210] * inv; w[210] = l;
      w[211] -= l * w[196];
      w[212] -= l * w[197];
      w[213] -= l * w[198];
      w[214] -= l * w[199];
      w[215] -= l * w[200];
      w[216] -= l * w[201];
    }
    { const R l = w[226] * inv; w[226] = l;
      w[227] -= l * w[196];
      w[228] -= l * w[197];
      w[229] -= l * w[198];
      w[230] -= l * w[199];
      w[231] -= l * w[200];
      w[232] -= l * w[201];
    }
    { const R l = w[245] * inv; w[245] = l;
      w[246] -= l * w[196];
      w[247] -= l * w[197];
      w[248] -= l * w[198];
      w[249] -= l * w[199];
      w[250] -= l * w[200];
      w[251] -= l * w[201];
    }
    { const R l = w[269] * inv; w[269] = l;
      w[270] -= l * w[196];
      w[271] -= l * w[197];
      w[272] -= l * w[198];
      w[273] -= l * w[199];
      w[274] -= l * w[200];
      w[275] -= l * w[201];
    }
    { const R l = w[289] * inv; w[289] = l;
      w[290] -= l * w[196];
      w[291] -= l * w[197];
      w[292] -= l * w[198];
      w[293] -= l * w[199];
      w[294] -= l * w[200];
      w[295] -= l * w[201];
    }
    { const R l = w[299] * inv; w[299] = l;
      w[300] -= l * w[196];
      w[301] -= l * w[197];
      w[302] -= l * w[198];
      w[303] -= l * w[199];
      w[304] -= l * w[200];
      w[305] -= l * w[201];
    }
  }
  {  // pivot 23: state 4 (S_bu), 5 rows x 5 cols
    const R pv = w[211];
    const R cm = fmax(fmax(fmax(fmax(fabs(w[227]), fabs(w[246])), fabs(w[270])), fabs(w[290])), fabs(w[300]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[23] = inv;
    { const R l = w[227] * inv; w[227] = l;
      w[228] -= l * w[212];
      w[229] -= l * w[213];
      w[230] -= l * w[214];
      w[231] -= l * w[215];
      w[232] -= l * w[216];
    }
    { const R l = w[246] * inv; w[246] = l;
      w[247] -= l * w[212];
      w[248] -= l * w[213];
      w[249] -= l * w[214];
      w[250] -= l * w[215];
      w[251] -= l * w[216];
    }
    { const R l = w[270] * inv; w[270] = l;
      w[271] -= l * w[212];
      w[272] -= l * w[213];
      w[273] -= l * w[214];
      w[274] -= l * w[215];
      w[275] -= l * w[216];
    }
    { const R l = w[290] * inv; w[290] = l;
      w[291] -= l * w[212];
      w[292] -= l * w[213];
      w[293] -= l * w[214];
      w[294] -= l * w[215];
      w[295] -= l * w[216];
    }
    { const R l = w[300] * inv; w[300] = l;
      w[301] -= l * w[212];
      w[302] -= l * w[213];
      w[303] -= l * w[214];
      w[304] -= l * w[215];
      w[305] -= l * w[216];
    }
  }
  {  // pivot 24: state 5 (S_pro), 4 rows x 4 cols
    const R pv = w[228];
    const R cm = fmax(fmax(fmax(fabs(w[247]), fabs(w[271])), fabs(w[291])), fabs(w[301]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[24] = inv;
    { const R l = w[247] * inv; w[247] = l;
      w[248] -= l * w[229];
      w[249] -= l * w[230];
      w[250] -= l * w[231];
      w[251] -= l * w[232];
    }
    { const R l = w[271] * inv; w[271] = l;
      w[272] -= l * w[229];
      w[273] -= l * w[230];
      w[274] -= l * w[231];
      w[275] -= l * w[232];
    }
    { const R l = w[291] * inv; w[291] = l;
      w[292] -= l * w[229];
      w[293] -= l * w[230];
      w[294] -= l * w[231];
      w[295] -= l * w[232];
    }
    { const R l = w[301] * inv; w[301] = l;
      w[302] -= l * w[229];
      w[303] -= l * w[230];
      w[304] -= l * w[231];
      w[305] -= l * w[232];
    }
  }
  {  // pivot 25: state 6 (S_ac), 3 rows x 3 cols
    const R pv = w[248];
    const R cm = fmax(fmax(fabs(w[272]), fabs(w[292])), fabs(w[302]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[25] = inv;
    { const R l = w[272] * inv; w[272] = l;
      w[273] -= l * w[249];
      w[274] -= l * w[250];
      w[275] -= l * w[251];
    }
    { const R l = w[292] * inv; w[292] = l;
      w[293] -= l * w[249];
      w[294] -= l * w[250];
      w[295] -= l * w[251];
    }
    { const R l = w[302] * inv; w[302] = l;
      w[303] -= l * w[249];
      w[304] -= l * w[250];
      w[305] -= l * w[251];
    }
  }
  {  // pivot 26: state 9 (S_IC), 2 rows x 2 cols
    const R pv = w[273];
    const R cm = fmax(fabs(w[293]), fabs(w[303]));
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[26] = inv;
    { const R l = w[293] * inv; w[293] = l;
      w[294] -= l * w[274];
      w[295] -= l * w[275];
    }
    { const R l = w[303] * inv; w[303] = l;
      w[304] -= l * w[274];
      w[305] -= l * w[275];
    }
  }
  {  // pivot 27: state 10 (S_IN), 1 rows x 1 cols
    const R pv = w[294];
    const R cm = fabs(w[304]);
    ok = ok && (fabs(pv) >= tau * cm);
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[27] = inv;
    { const R l = w[304] * inv; w[304] = l;
      w[305] -= l * w[295];
    }
  }
  {  // pivot 28: state 17 (X_aa), 0 rows x 0 cols
    const R pv = w[305];
    ok = ok && (pv != R(0)) && isfinite(pv);
    const R inv = rcp<R>(pv);
    dinv[28] = inv;
  }
  return ok;
}

// Solve W x = b in place (b indexed by state).
template <class R>
CHAD_HD void solve(const R* w, const R* dinv, R* b) {
  R z0 = b[11];
  R z1 = b[23];
  R z2 = b[24];
  R z3 = b[25];
  R z4 = b[13];
  R z5 = b[14];
  R z6 = b[15];
  R z7 = b[26];
  R z8 = b[27];
  R z9 = b[8];
  R z10 = b[28];
  R z11 = b[22];
  R z12 = b[21];
  R z13 = b[20];
  R z14 = b[2];
  R z15 = b[18];
  R z16 = b[0];
  R z17 = b[16];
  R z18 = b[19];
  R z19 = b[12];
  R z20 = b[7];
  R z21 = b[1];
  R z22 = b[3];
  R z23 = b[4];
  R z24 = b[5];
  R z25 = b[6];
  R z26 = b[9];
  R z27 = b[10];
  R z28 = b[17];
  z8 -= w[16] * z7;
  z9 -= w[21] * z2;
  z9 -= w[22] * z3;
  z9 -= w[23] * z8;
  z10 -= w[35] * z2;
  z10 -= w[36] * z3;
  z10 -= w[37] * z7;
  z10 -= w[38] * z8;
  z10 -= w[39] * z9;
  z11 -= w[50] * z2;
  z11 -= w[51] * z3;
  z12 -= w[60] * z2;
  z12 -= w[61] * z3;
  z13 -= w[69] * z2;
  z13 -= w[70] * z3;
  z14 -= w[79] * z2;
  z14 -= w[80] * z3;
  z14 -= w[81] * z6;
  z15 -= w[92] * z2;
  z15 -= w[93] * z3;
  z15 -= w[94] * z14;
  z16 -= w[104] * z2;
  z16 -= w[105] * z3;
  z16 -= w[106] * z4;
  z16 -= w[107] * z6;
  z17 -= w[117] * z2;
  z17 -= w[118] * z3;
  z17 -= w[119] * z16;
  z18 -= w[128] * z2;
  z18 -= w[129] * z3;
  z19 -= w[138] * z11;
  z19 -= w[139] * z12;
  z19 -= w[140] * z13;
  z19 -= w[141] * z15;
  z19 -= w[142] * z17;
  z19 -= w[143] * z18;
  z20 -= w[153] * z2;
  z20 -= w[154] * z3;
  z20 -= w[155] * z7;
  z20 -= w[156] * z8;
  z20 -= w[157] * z9;
  z20 -= w[158] * z10;
  z20 -= w[159] * z11;
  z20 -= w[160] * z12;
  z20 -= w[161] * z13;
  z20 -= w[162] * z14;
  z20 -= w[163] * z15;
  z20 -= w[164] * z16;
  z20 -= w[165] * z17;
  z20 -= w[166] * z18;
  z20 -= w[167] * z19;
  z21 -= w[177] * z2;
  z21 -= w[178] * z3;
  z21 -= w[179] * z5;
  z21 -= w[180] * z19;
  z21 -= w[181] * z20;
  z22 -= w[190] * z2;
  z22 -= w[191] * z3;
  z22 -= w[192] * z18;
  z22 -= w[193] * z20;
  z22 -= w[194] * z21;
  z23 -= w[202] * z2;
  z23 -= w[203] * z3;
  z23 -= w[204] * z16;
  z23 -= w[205] * z17;
  z23 -= w[206] * z18;
  z23 -= w[207] * z19;
  z23 -= w[208] * z20;
  z23 -= w[209] * z21;
  z23 -= w[210] * z22;
  z24 -= w[217] * z2;
  z24 -= w[218] * z3;
  z24 -= w[219] * z13;
  z24 -= w[220] * z16;
  z24 -= w[221] * z17;
  z24 -= w[222] * z18;
  z24 -= w[223] * z19;
  z24 -= w[224] * z20;
  z24 -= w[225] * z21;
  z24 -= w[226] * z22;
  z24 -= w[227] * z23;
  z25 -= w[233] * z2;
  z25 -= w[234] * z3;
  z25 -= w[235] * z12;
  z25 -= w[236] * z13;
  z25 -= w[237] * z14;
  z25 -= w[238] * z15;
  z25 -= w[239] * z16;
  z25 -= w[240] * z17;
  z25 -= w[241] * z18;
  z25 -= w[242] * z19;
  z25 -= w[243] * z20;
  z25 -= w[244] * z21;
  z25 -= w[245] * z22;
  z25 -= w[246] * z23;
  z25 -= w[247] * z24;
  z26 -= w[252] * z2;
  z26 -= w[253] * z3;
  z26 -= w[254] * z4;
  z26 -= w[255] * z5;
  z26 -= w[256] * z6;
  z26 -= w[257] * z10;
  z26 -= w[258] * z11;
  z26 -= w[259] * z12;
  z26 -= w[260] * z13;
  z26 -= w[261] * z14;
  z26 -= w[262] * z15;
  z26 -= w[263] * z16;
  z26 -= w[264] * z17;
  z26 -= w[265] * z18;
  z26 -= w[266] * z19;
  z26 -= w[267] * z20;
  z26 -= w[268] * z21;
  z26 -= w[269] * z22;
  z26 -= w[270] * z23;
  z26 -= w[271] * z24;
  z26 -= w[272] * z25;
  z27 -= w[276] * z2;
  z27 -= w[277] * z3;
  z27 -= w[278] * z11;
  z27 -= w[279] * z12;
  z27 -= w[280] * z13;
  z27 -= w[281] * z14;
  z27 -= w[282] * z15;
  z27 -= w[283] * z16;
  z27 -= w[284] * z17;
  z27 -= w[285] * z18;
  z27 -= w[286] * z19;
  z27 -= w[287] * z20;
  z27 -= w[288] * z21;
  z27 -= w[289] * z22;
  z27 -= w[290] * z23;
  z27 -= w[291] * z24;
  z27 -= w[292] * z25;
  z27 -= w[293] * z26;
  z28 -= w[296] * z2;
  z28 -= w[297] * z3;
  z28 -= w[298] * z21;
  z28 -= w[299] * z22;
  z28 -= w[300] * z23;
  z28 -= w[301] * z24;
  z28 -= w[302] * z25;
  z28 -= w[303] * z26;
  z28 -= w[304] * z27;
  z28 *= dinv[28];
  z27 -= w[295] * z28;
  z27 *= dinv[27];
  z26 -= w[274] * z27;
  z26 -= w[275] * z28;
  z26 *= dinv[26];
  z25 -= w[249] * z26;
  z25 -= w[250] * z27;
  z25 -= w[251] * z28;
  z25 *= dinv[25];
  z24 -= w[229] * z25;
  z24 -= w[230] * z26;
  z24 -= w[231] * z27;
  z24 -= w[232] * z28;
  z24 *= dinv[24];
  z23 -= w[212] * z24;
  z23 -= w[213] * z25;
  z23 -= w[214] * z26;
  z23 -= w[215] * z27;
  z23 -= w[216] * z28;
  z23 *= dinv[23];
  z22 -= w[196] * z23;
  z22 -= w[197] * z24;
  z22 -= w[198] * z25;
  z22 -= w[199] * z26;
  z22 -= w[200] * z27;
  z22 -= w[201] * z28;
  z22 *= dinv[22];
  z21 -= w[183] * z22;
  z21 -= w[184] * z23;
  z21 -= w[185] * z24;
  z21 -= w[186] * z25;
  z21 -= w[187] * z26;
  z21 -= w[188] * z27;
  z21 -= w[189] * z28;
  z21 *= dinv[21];
  z20 -= w[169] * z21;
  z20 -= w[170] * z22;
  z20 -= w[171] * z23;
  z20 -= w[172] * z24;
  z20 -= w[173] * z25;
  z20 -= w[174] * z26;
  z20 -= w[175] * z27;
  z20 -= w[176] * z28;
  z20 *= dinv[20];
  z19 -= w[145] * z20;
  z19 -= w[146] * z22;
  z19 -= w[147] * z23;
  z19 -= w[148] * z24;
  z19 -= w[149] * z25;
  z19 -= w[150] * z26;
  z19 -= w[151] * z27;
  z19 -= w[152] * z28;
  z19 *= dinv[19];
  z18 -= w[131] * z20;
  z18 -= w[132] * z22;
  z18 -= w[133] * z23;
  z18 -= w[134] * z24;
  z18 -= w[135] * z25;
  z18 -= w[136] * z26;
  z18 -= w[137] * z27;
  z18 *= dinv[18];
  z17 -= w[121] * z19;
  z17 -= w[122] * z22;
  z17 -= w[123] * z23;
  z17 -= w[124] * z24;
  z17 -= w[125] * z25;
  z17 -= w[126] * z26;
  z17 -= w[127] * z27;
  z17 *= dinv[17];
  z16 -= w[109] * z17;
  z16 -= w[110] * z19;
  z16 -= w[111] * z22;
  z16 -= w[112] * z23;
  z16 -= w[113] * z24;
  z16 -= w[114] * z25;
  z16 -= w[115] * z26;
  z16 -= w[116] * z27;
  z16 *= dinv[16];
  z15 -= w[96] * z19;
  z15 -= w[97] * z20;
  z15 -= w[98] * z22;
  z15 -= w[99] * z23;
  z15 -= w[100] * z24;
  z15 -= w[101] * z25;
  z15 -= w[102] * z26;
  z15 -= w[103] * z27;
  z15 *= dinv[15];
  z14 -= w[83] * z15;
  z14 -= w[84] * z19;
  z14 -= w[85] * z20;
  z14 -= w[86] * z22;
  z14 -= w[87] * z23;
  z14 -= w[88] * z24;
  z14 -= w[89] * z25;
  z14 -= w[90] * z26;
  z14 -= w[91] * z27;
  z14 *= dinv[14];
  z13 -= w[72] * z20;
  z13 -= w[73] * z22;
  z13 -= w[74] * z23;
  z13 -= w[75] * z24;
  z13 -= w[76] * z25;
  z13 -= w[77] * z26;
  z13 -= w[78] * z27;
  z13 *= dinv[13];
  z12 -= w[63] * z22;
  z12 -= w[64] * z23;
  z12 -= w[65] * z24;
  z12 -= w[66] * z25;
  z12 -= w[67] * z26;
  z12 -= w[68] * z27;
  z12 *= dinv[12];
  z11 -= w[53] * z20;
  z11 -= w[54] * z22;
  z11 -= w[55] * z23;
  z11 -= w[56] * z24;
  z11 -= w[57] * z25;
  z11 -= w[58] * z26;
  z11 -= w[59] * z27;
  z11 *= dinv[11];
  z10 -= w[41] * z11;
  z10 -= w[42] * z12;
  z10 -= w[43] * z20;
  z10 -= w[44] * z22;
  z10 -= w[45] * z23;
  z10 -= w[46] * z24;
  z10 -= w[47] * z25;
  z10 -= w[48] * z26;
  z10 -= w[49] * z27;
  z10 *= dinv[10];
  z9 -= w[25] * z10;
  z9 -= w[26] * z11;
  z9 -= w[27] * z12;
  z9 -= w[28] * z20;
  z9 -= w[29] * z22;
  z9 -= w[30] * z23;
  z9 -= w[31] * z24;
  z9 -= w[32] * z25;
  z9 -= w[33] * z26;
  z9 -= w[34] * z27;
  z9 *= dinv[9];
  z8 -= w[18] * z9;
  z8 -= w[19] * z10;
  z8 -= w[20] * z20;
  z8 *= dinv[8];
  z7 -= w[13] * z8;
  z7 -= w[14] * z10;
  z7 -= w[15] * z20;
  z7 *= dinv[7];
  z6 -= w[11] * z19;
  z6 *= dinv[6];
  z5 -= w[9] * z19;
  z5 *= dinv[5];
  z4 -= w[7] * z19;
  z4 *= dinv[4];
  z3 *= dinv[3];
  z2 *= dinv[2];
  z1 -= w[3] * z19;
  z1 *= dinv[1];
  z0 -= w[1] * z19;
  z0 *= dinv[0];
  b[11] = z0;
  b[23] = z1;
  b[24] = z2;
  b[25] = z3;
  b[13] = z4;
  b[14] = z5;
  b[15] = z6;
  b[26] = z7;
  b[27] = z8;
  b[8] = z9;
  b[28] = z10;
  b[22] = z11;
  b[21] = z12;
  b[20] = z13;
  b[2] = z14;
  b[18] = z15;
  b[0] = z16;
  b[16] = z17;
  b[19] = z18;
  b[12] = z19;
  b[7] = z20;
  b[1] = z21;
  b[3] = z22;
  b[4] = z23;
  b[5] = z24;
  b[6] = z25;
  b[9] = z26;
  b[10] = z27;
  b[17] = z28;
}

// out = J x over the structural nonzeros of J (slots of a J array).
template <class RJ>
CHAD_HD void jx(const RJ* j, const double* x, double* out) {
  out[0] = double(j[108]) * x[0] + double(j[111]) * x[3] + double(j[112]) * x[4] + double(j[113]) * x[5] + double(j[114]) * x[6] + double(j[115]) * x[9] + double(j[116]) * x[10] + double(j[106]) * x[13] + double(j[107]) * x[15] + double(j[109]) * x[16] + double(j[104]) * x[24] + double(j[105]) * x[25];
  out[1] = double(j[182]) * x[1] + double(j[183]) * x[3] + double(j[184]) * x[4] + double(j[185]) * x[5] + double(j[186]) * x[6] + double(j[187]) * x[9] + double(j[188]) * x[10] + double(j[179]) * x[14] + double(j[189]) * x[17] + double(j[177]) * x[24] + double(j[178]) * x[25];
  out[2] = double(j[82]) * x[2] + double(j[86]) * x[3] + double(j[87]) * x[4] + double(j[88]) * x[5] + double(j[89]) * x[6] + double(j[85]) * x[7] + double(j[90]) * x[9] + double(j[91]) * x[10] + double(j[81]) * x[15] + double(j[83]) * x[18] + double(j[79]) * x[24] + double(j[80]) * x[25];
  out[3] = double(j[194]) * x[1] + double(j[195]) * x[3] + double(j[196]) * x[4] + double(j[197]) * x[5] + double(j[198]) * x[6] + double(j[193]) * x[7] + double(j[199]) * x[9] + double(j[200]) * x[10] + double(j[201]) * x[17] + double(j[192]) * x[19] + double(j[190]) * x[24] + double(j[191]) * x[25];
  out[4] = double(j[204]) * x[0] + double(j[209]) * x[1] + double(j[210]) * x[3] + double(j[211]) * x[4] + double(j[212]) * x[5] + double(j[213]) * x[6] + double(j[208]) * x[7] + double(j[214]) * x[9] + double(j[215]) * x[10] + double(j[205]) * x[16] + double(j[216]) * x[17] + double(j[206]) * x[19] + double(j[202]) * x[24] + double(j[203]) * x[25];
  out[5] = double(j[220]) * x[0] + double(j[225]) * x[1] + double(j[226]) * x[3] + double(j[227]) * x[4] + double(j[228]) * x[5] + double(j[229]) * x[6] + double(j[224]) * x[7] + double(j[230]) * x[9] + double(j[231]) * x[10] + double(j[221]) * x[16] + double(j[232]) * x[17] + double(j[222]) * x[19] + double(j[219]) * x[20] + double(j[217]) * x[24] + double(j[218]) * x[25];
  out[6] = double(j[239]) * x[0] + double(j[244]) * x[1] + double(j[237]) * x[2] + double(j[245]) * x[3] + double(j[246]) * x[4] + double(j[247]) * x[5] + double(j[248]) * x[6] + double(j[243]) * x[7] + double(j[249]) * x[9] + double(j[250]) * x[10] + double(j[240]) * x[16] + double(j[251]) * x[17] + double(j[238]) * x[18] + double(j[241]) * x[19] + double(j[236]) * x[20] + double(j[235]) * x[21] + double(j[233]) * x[24] + double(j[234]) * x[25];
  out[7] = double(j[164]) * x[0] + double(j[169]) * x[1] + double(j[162]) * x[2] + double(j[170]) * x[3] + double(j[171]) * x[4] + double(j[172]) * x[5] + double(j[173]) * x[6] + double(j[168]) * x[7] + double(j[174]) * x[9] + double(j[175]) * x[10] + double(j[165]) * x[16] + double(j[176]) * x[17] + double(j[163]) * x[18] + double(j[166]) * x[19] + double(j[161]) * x[20] + double(j[159]) * x[22] + double(j[153]) * x[24] + double(j[154]) * x[25] + double(j[155]) * x[26];
  out[8] = double(j[29]) * x[3] + double(j[30]) * x[4] + double(j[31]) * x[5] + double(j[32]) * x[6] + double(j[28]) * x[7] + double(j[24]) * x[8] + double(j[33]) * x[9] + double(j[34]) * x[10] + double(j[27]) * x[21] + double(j[26]) * x[22] + double(j[21]) * x[24] + double(j[22]) * x[25] + double(j[23]) * x[27];
  out[9] = double(j[263]) * x[0] + double(j[268]) * x[1] + double(j[261]) * x[2] + double(j[269]) * x[3] + double(j[270]) * x[4] + double(j[271]) * x[5] + double(j[272]) * x[6] + double(j[267]) * x[7] + double(j[273]) * x[9] + double(j[274]) * x[10] + double(j[266]) * x[12] + double(j[254]) * x[13] + double(j[255]) * x[14] + double(j[256]) * x[15] + double(j[264]) * x[16] + double(j[275]) * x[17] + double(j[262]) * x[18] + double(j[265]) * x[19] + double(j[260]) * x[20] + double(j[259]) * x[21] + double(j[258]) * x[22] + double(j[252]) * x[24] + double(j[253]) * x[25] + double(j[257]) * x[28];
  out[10] = double(j[283]) * x[0] + double(j[288]) * x[1] + double(j[281]) * x[2] + double(j[289]) * x[3] + double(j[290]) * x[4] + double(j[291]) * x[5] + double(j[292]) * x[6] + double(j[287]) * x[7] + double(j[293]) * x[9] + double(j[294]) * x[10] + double(j[286]) * x[12] + double(j[284]) * x[16] + double(j[295]) * x[17] + double(j[282]) * x[18] + double(j[285]) * x[19] + double(j[280]) * x[20] + double(j[279]) * x[21] + double(j[278]) * x[22] + double(j[276]) * x[24] + double(j[277]) * x[25];
  out[11] = double(j[0]) * x[11] + double(j[1]) * x[12];
  out[12] = double(j[144]) * x[12] + double(j[142]) * x[16] + double(j[152]) * x[17] + double(j[141]) * x[18] + double(j[143]) * x[19] + double(j[140]) * x[20] + double(j[139]) * x[21] + double(j[138]) * x[22];
  out[13] = double(j[7]) * x[12] + double(j[6]) * x[13];
  out[14] = double(j[9]) * x[12] + double(j[8]) * x[14];
  out[15] = double(j[11]) * x[12] + double(j[10]) * x[15];
  out[16] = double(j[119]) * x[0] + double(j[122]) * x[3] + double(j[123]) * x[4] + double(j[124]) * x[5] + double(j[125]) * x[6] + double(j[126]) * x[9] + double(j[127]) * x[10] + double(j[120]) * x[16] + double(j[117]) * x[24] + double(j[118]) * x[25];
  out[17] = double(j[298]) * x[1] + double(j[299]) * x[3] + double(j[300]) * x[4] + double(j[301]) * x[5] + double(j[302]) * x[6] + double(j[303]) * x[9] + double(j[304]) * x[10] + double(j[305]) * x[17] + double(j[296]) * x[24] + double(j[297]) * x[25];
  out[18] = double(j[94]) * x[2] + double(j[98]) * x[3] + double(j[99]) * x[4] + double(j[100]) * x[5] + double(j[101]) * x[6] + double(j[97]) * x[7] + double(j[102]) * x[9] + double(j[103]) * x[10] + double(j[95]) * x[18] + double(j[92]) * x[24] + double(j[93]) * x[25];
  out[19] = double(j[132]) * x[3] + double(j[133]) * x[4] + double(j[134]) * x[5] + double(j[135]) * x[6] + double(j[131]) * x[7] + double(j[136]) * x[9] + double(j[137]) * x[10] + double(j[130]) * x[19] + double(j[128]) * x[24] + double(j[129]) * x[25];
  out[20] = double(j[73]) * x[3] + double(j[74]) * x[4] + double(j[75]) * x[5] + double(j[76]) * x[6] + double(j[72]) * x[7] + double(j[77]) * x[9] + double(j[78]) * x[10] + double(j[71]) * x[20] + double(j[69]) * x[24] + double(j[70]) * x[25];
  out[21] = double(j[63]) * x[3] + double(j[64]) * x[4] + double(j[65]) * x[5] + double(j[66]) * x[6] + double(j[67]) * x[9] + double(j[68]) * x[10] + double(j[62]) * x[21] + double(j[60]) * x[24] + double(j[61]) * x[25];
  out[22] = double(j[54]) * x[3] + double(j[55]) * x[4] + double(j[56]) * x[5] + double(j[57]) * x[6] + double(j[53]) * x[7] + double(j[58]) * x[9] + double(j[59]) * x[10] + double(j[52]) * x[22] + double(j[50]) * x[24] + double(j[51]) * x[25];
  out[23] = double(j[3]) * x[12] + double(j[2]) * x[23];
  out[24] = double(j[4]) * x[24];
  out[25] = double(j[5]) * x[25];
  out[26] = double(j[15]) * x[7] + double(j[12]) * x[26] + double(j[13]) * x[27] + double(j[14]) * x[28];
  out[27] = double(j[18]) * x[8] + double(j[16]) * x[26] + double(j[17]) * x[27] + double(j[19]) * x[28];
  out[28] = double(j[44]) * x[3] + double(j[45]) * x[4] + double(j[46]) * x[5] + double(j[47]) * x[6] + double(j[48]) * x[9] + double(j[49]) * x[10] + double(j[35]) * x[24] + double(j[36]) * x[25] + double(j[37]) * x[26] + double(j[38]) * x[27] + double(j[40]) * x[28];
}

constexpr int kFactorFlops = 1495;
constexpr int kSolveFlops = 583;
constexpr int kJxFlops = 558;

}  // namespace sp
}  // namespace chad
