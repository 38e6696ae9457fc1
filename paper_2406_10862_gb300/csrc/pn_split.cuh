// The explicit black-oil phase split of Sec. 2.1: from the pressure and the
// component amounts per bulk volume (surface volumes) to the fluid volumes,
// the saturations and the natural variables (p, S_w[, X]), with derivatives
// by (P, N_w, N_o[, N_g]).  Used by the (P, N) Newton path and by IMPEC.
#pragma once

#include "ocp_internal.cuh"

namespace ocp {

template <int NB>
struct Split {
  int flag;                 // 1: all gas dissolved (undersaturated oil)
  double sw, x;             // natural variables besides p (x = S_g or R_s)
  double Vf;                // fluid volume per bulk volume
  double dVf[NB + 1];       // d V_f / d (P, N_w, N_o[, N_g])
  double M[NB][NB + 1];     // d (p, S_w[, X]) / d (P, N_w, N_o[, N_g])
};

template <int NB>
__device__ __forceinline__ void phase_split(const Params& P, const Table& T, double p, double nw, double no,
                                            double ng, Split<NB>& out) {
  constexpr int L = NB + 1;
  int f = 0;
  double x_pvt = 0.0;
  if (NB == 3) {
    Pvt s0;
    pvt<3, false>(P, T, p, 0.0, 0, s0);           // R_s,sat(p)
    if (positive(no) && ng <= s0.rs * no) {
      f = 1;
      x_pvt = ng / no;
    }
  }
  Pvt v;
  pvt<NB, false>(P, T, p, x_pvt, f, v);
  double dVw[L] = {}, dVo[L] = {}, dVg[L] = {}, dRs[L] = {};
  const double ibw = 1.0 / v.bw;
  const double Vw = nw * ibw;
  dVw[0] = -Vw * v.bw_p * ibw;
  dVw[1] = ibw;
  const double ibo = 1.0 / v.bo;
  const double Vo = no * ibo;
  double Vg = 0.0;
  dVo[0] = -Vo * v.bo_p * ibo;
  if (NB == 3 && f == 1) {
    const double ino = 1.0 / no;
    dRs[2] = -x_pvt * ino;
    dRs[3] = ino;
    dVo[2] = ibo - Vo * v.bo_x * dRs[2] * ibo;
    dVo[3] = -Vo * v.bo_x * dRs[3] * ibo;
  } else {
    dVo[2] = ibo;
    if (NB == 3) {
      const double ibg = 1.0 / v.bg;
      Vg = fma(-v.rs, no, ng) * ibg;
      dVg[0] = fma(-v.rs_p, no, -Vg * v.bg_p) * ibg;
      dVg[2] = -v.rs * ibg;
      dVg[3] = ibg;
    }
  }
  out.flag = f;
  out.Vf = Vw + Vo + Vg;
  const double iVf = 1.0 / out.Vf;
  for (int k = 0; k < L; ++k) out.dVf[k] = dVw[k] + dVo[k] + dVg[k];
  out.sw = Vw * iVf;
  for (int k = 0; k < L; ++k) {
    out.M[0][k] = (k == 0) ? 1.0 : 0.0;
    out.M[1][k] = (dVw[k] - out.sw * out.dVf[k]) * iVf;
  }
  out.x = 0.0;
  if (NB == 3) {
    if (f == 1) {
      out.x = x_pvt;
      for (int k = 0; k < L; ++k) out.M[2][k] = dRs[k];
    } else {
      out.x = Vg * iVf;
      for (int k = 0; k < L; ++k) out.M[2][k] = (dVg[k] - out.x * out.dVf[k]) * iVf;
    }
  }
}

}  // namespace ocp
