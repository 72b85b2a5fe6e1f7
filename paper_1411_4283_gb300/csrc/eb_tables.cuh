// Monomial, shift and footprint tables used by the build kernels.
//
// Interpolant monomials: multi-indices p with |p| <= Q (Sec. 2.2: |p| < P,
// P = Q + 1), graded order (degree 0, then for each degree q the exponents
// with p0 from q down to 0, p1 from q - p0 down to 0, ...).  The same order
// indexes the stored moment tables, so the first K stored moments are the
// moments of degree <= Q.
#pragma once
#include <stdint.h>

#include "eb_internal.cuh"

namespace eb {

constexpr int MAXD = 3;
constexpr int MAXLN = 5;    // monomials on one line of the shift (exponents 0..4)

struct Tables {
  int dim, K, KS, KFS;
  int8_t mon[MAXK][3];          // exponents of monomial i
  // separable moment shift along d: the monomials whose other exponents agree form a line
  // ln_idx[d][l][0..ln_len-1] ordered by the exponent along d (0, 1, ...); the shifted moments of a
  // line are m'_p = sum_{j <= p} C(p, j) delta^(p-j) m_j, evaluated by repeated synthetic steps
  int nln[MAXD];
  uint8_t ln_len[MAXD][MAXK];
  uint8_t ln_idx[MAXD][MAXK][MAXLN];
  // lower[d][i] = index of p_i - e_d (or -1 when p_d = 0)
  int8_t lower[MAXD][MAXK];
  // tangential map for faces normal to d: tang[d][i] = index of p_t in the (D-1)-dim stored
  // face table when p_d == 0, else -1
  int16_t tang[MAXD][MAXK];
  // closed-form moments of a full cell and of a full face normal to d (embedded in D dims)
  double full_vol[MAXK];
  double full_face[MAXD][MAXK];
};

// host builder (eb_api.cu)
bool make_tables(int dim, int order, int mdeg, Tables* t);

// ---------------------------------------------------------------- footprint
// Operator footprint of a cell for radius R and box neighbourhoods: offsets
// with |d|_inf <= R, plus offsets with exactly one |d_k| = R+1 and the others
// <= R (union of the neighbourhood boxes of the cell's faces).  Path
// neighbourhoods use the L1 ball of radius R+1.  Canonical order: z-major.
struct Foot {
  int n;
  int R, dim, box;
  int8_t d[MAX_FOOT][3];
};

__host__ __device__ inline bool in_footprint(int dx, int dy, int dz, int R, int box) {
  int ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
  if (!box) return ax + ay + az <= R + 1;
  int over = (ax > R) + (ay > R) + (az > R);
  int mx = ax > ay ? (ax > az ? ax : az) : (ay > az ? ay : az);
  return mx <= R + 1 && over <= 1;
}

}  // namespace eb
