// D3Q27 lattice and moment transforms used by the kernels.
//
// Velocities are held in tensor order t = (cx+1) + 3(cy+1) + 9(cz+1), so the
// rest velocity is t = 13 and the opposite of t is 26 - t.  The D3Q27 weights
// of Sec. II are the products of the D1Q3 weights (1/6, 2/3, 1/6) of the three
// components.  The paper's own direction order (Eq. velSet, fixed by rows 2-4
// of the printed M in App. A) is used only at the C ABI.
//
// Moments.  The raw moments R_abc = sum_i cx^a cy^b cz^c f_i (a,b,c in 0..2)
// follow from three one-dimensional 3-point transforms (one per axis).  The
// moments m_1..m_27 of Eq. (momentSet) are sparse integer combinations of the
// R_abc (moment_forward).  Because the rows of M are mutually orthogonal,
// M^-1 = M^T diag(1/|M_j|^2), so the way back is the transpose of the same two
// steps (moment_adjoint, then the transposed 1D transforms) scaled by the
// inverse row norms; the kernels never hold a dense 27x27 matrix.
#pragma once
#include <stdint.h>

namespace lbmk {

constexpr int Q = 27;
constexpr int REST = 13;

__host__ __device__ constexpr int cx_of(int t) { return t % 3 - 1; }
__host__ __device__ constexpr int cy_of(int t) { return (t / 3) % 3 - 1; }
__host__ __device__ constexpr int cz_of(int t) { return t / 9 - 1; }
__host__ __device__ constexpr int opp_of(int t) { return 26 - t; }
__host__ __device__ constexpr int tensor_index(int cx, int cy, int cz) { return (cx + 1) + 3 * (cy + 1) + 9 * (cz + 1); }
__host__ __device__ constexpr int speed2_of(int t) {
  return cx_of(t) * cx_of(t) + cy_of(t) * cy_of(t) + cz_of(t) * cz_of(t);
}
__host__ __device__ constexpr double w1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
// D3Q27 weight w_i (Sec. II): 8/27, 2/27, 1/54, 1/216 by |c|^2 = 0, 1, 2, 3.
__host__ __device__ constexpr double weight_of(int t) { return w1d(cx_of(t)) * w1d(cy_of(t)) * w1d(cz_of(t)); }

// Paper direction i (0-based, i.e. the paper's i-1) -> tensor index.
// Eq. (velSet) gives the groups; the order inside each group is the one of
// rows 2-4 (c_x, c_y, c_z) of the transformation matrix printed in App. A.
__host__ __device__ inline int paper_to_tensor(int i) {
  switch (i) {
    case 0: return tensor_index(0, 0, 0);
    case 1: return tensor_index(1, 0, 0);
    case 2: return tensor_index(-1, 0, 0);
    case 3: return tensor_index(0, 1, 0);
    case 4: return tensor_index(0, -1, 0);
    case 5: return tensor_index(0, 0, 1);
    case 6: return tensor_index(0, 0, -1);
    case 7: return tensor_index(1, 1, 0);
    case 8: return tensor_index(-1, -1, 0);
    case 9: return tensor_index(1, -1, 0);
    case 10: return tensor_index(-1, 1, 0);
    case 11: return tensor_index(0, 1, 1);
    case 12: return tensor_index(0, -1, -1);
    case 13: return tensor_index(0, 1, -1);
    case 14: return tensor_index(0, -1, 1);
    case 15: return tensor_index(1, 0, 1);
    case 16: return tensor_index(-1, 0, -1);
    case 17: return tensor_index(-1, 0, 1);
    case 18: return tensor_index(1, 0, -1);
    case 19: return tensor_index(1, 1, 1);
    case 20: return tensor_index(-1, -1, -1);
    case 21: return tensor_index(1, 1, -1);
    case 22: return tensor_index(-1, -1, 1);
    case 23: return tensor_index(-1, 1, 1);
    case 24: return tensor_index(1, -1, -1);
    case 25: return tensor_index(1, -1, 1);
    default: return tensor_index(-1, 1, -1);
  }
}

// Relaxation slot of moment j (0-based) in K = diag[s1 x4, s5, s6 x2, s8 x3,
// s11 x3, s14 x3, s17, s18, s19 x2, s21 x3, s24 x3, s27] (Sec. II).
__host__ __device__ inline int kslot_of(int j) {
  if (j < 4) return 1;
  if (j == 4) return 5;
  if (j < 7) return 6;
  if (j < 10) return 8;
  if (j < 13) return 11;
  if (j < 16) return 14;
  if (j == 16) return 17;
  if (j == 17) return 18;
  if (j < 20) return 19;
  if (j < 23) return 21;
  if (j < 26) return 24;
  return 27;
}

// ---------------------------------------------------------------------------
// raw moments: in-place 1D 3-point transforms along x, y and z.
// (f_-, f_0, f_+) -> (f_- + f_0 + f_+, f_+ - f_-, f_+ + f_-): orders 0, 1, 2.
template <typename R>
__host__ __device__ __forceinline__ void tri_forward(R& a, R& b, R& c) {
  R s = c + a, d = c - a;
  a = s + b;
  b = d;
  c = s;
}
// transpose of tri_forward: (k0, k1, k2) -> (k0 - k1 + k2, k0, k0 + k1 + k2).
template <typename R>
__host__ __device__ __forceinline__ void tri_adjoint(R& a, R& b, R& c) {
  R k0 = a, k1 = b, k2 = c;
  R s = k0 + k2;
  a = s - k1;
  b = k0;
  c = s + k1;
}

template <typename R>
__host__ __device__ __forceinline__ void raw_forward(R v[27]) {
#pragma unroll
  for (int l = 0; l < 9; ++l) tri_forward(v[3 * l + 0], v[3 * l + 1], v[3 * l + 2]);  // x
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    int base = (l % 3) + 9 * (l / 3);
    tri_forward(v[base], v[base + 3], v[base + 6]);  // y
  }
#pragma unroll
  for (int l = 0; l < 9; ++l) tri_forward(v[l], v[l + 9], v[l + 18]);  // z
}

template <typename R>
__host__ __device__ __forceinline__ void raw_adjoint(R v[27]) {
#pragma unroll
  for (int l = 0; l < 9; ++l) tri_adjoint(v[l], v[l + 9], v[l + 18]);
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    int base = (l % 3) + 9 * (l / 3);
    tri_adjoint(v[base], v[base + 3], v[base + 6]);
  }
#pragma unroll
  for (int l = 0; l < 9; ++l) tri_adjoint(v[3 * l + 0], v[3 * l + 1], v[3 * l + 2]);
}

#define LBMK_R(a, b, c) r[(a) + 3 * (b) + 9 * (c)]

// Moments 5..27 of Eq. (momentSet) (0-based m[4..26]) from the raw moments.
// Moments 1..4 (density and momentum) are conserved and not needed here.
template <typename R>
__host__ __device__ __forceinline__ void moment_forward(const R r[27], R m[27]) {
  const R S2 = LBMK_R(2, 0, 0) + LBMK_R(0, 2, 0) + LBMK_R(0, 0, 2);
  const R S4 = LBMK_R(2, 2, 0) + LBMK_R(0, 2, 2) + LBMK_R(2, 0, 2);
  m[0] = LBMK_R(0, 0, 0);
  m[1] = LBMK_R(1, 0, 0);
  m[2] = LBMK_R(0, 1, 0);
  m[3] = LBMK_R(0, 0, 1);
  m[4] = S2 - R(2) * LBMK_R(0, 0, 0);                                        // -2<1> + <|c|^2>
  m[5] = R(2) * LBMK_R(2, 0, 0) - LBMK_R(0, 2, 0) - LBMK_R(0, 0, 2);        // 2<cx^2> - <cy^2+cz^2>
  m[6] = LBMK_R(0, 2, 0) - LBMK_R(0, 0, 2);                                  // <cy^2 - cz^2>
  m[7] = LBMK_R(1, 1, 0);                                                    // <cx cy>
  m[8] = LBMK_R(0, 1, 1);                                                    // <cy cz>
  m[9] = LBMK_R(1, 0, 1);                                                    // <cz cx>
  m[10] = R(3) * (LBMK_R(1, 2, 0) + LBMK_R(1, 0, 2)) - R(4) * LBMK_R(1, 0, 0);
  m[11] = R(3) * (LBMK_R(0, 1, 2) + LBMK_R(2, 1, 0)) - R(4) * LBMK_R(0, 1, 0);
  m[12] = R(3) * (LBMK_R(2, 0, 1) + LBMK_R(0, 2, 1)) - R(4) * LBMK_R(0, 0, 1);
  m[13] = R(4) * LBMK_R(1, 0, 0) - R(6) * (LBMK_R(1, 2, 0) + LBMK_R(1, 0, 2)) + R(9) * LBMK_R(1, 2, 2);
  m[14] = R(4) * LBMK_R(0, 1, 0) - R(6) * (LBMK_R(0, 1, 2) + LBMK_R(2, 1, 0)) + R(9) * LBMK_R(2, 1, 2);
  m[15] = R(4) * LBMK_R(0, 0, 1) - R(6) * (LBMK_R(2, 0, 1) + LBMK_R(0, 2, 1)) + R(9) * LBMK_R(2, 2, 1);
  m[16] = R(4) * (LBMK_R(0, 0, 0) - S2) + R(3) * S4;                                         // 4<1-|c|^2> + 3<..>
  m[17] = R(-8) * LBMK_R(0, 0, 0) + R(12) * S2 - R(18) * S4 + R(27) * LBMK_R(2, 2, 2);
  m[18] = R(2) * (LBMK_R(0, 0, 2) + LBMK_R(0, 2, 0)) + R(3) * (LBMK_R(2, 2, 0) + LBMK_R(2, 0, 2)) -
          R(4) * LBMK_R(2, 0, 0) - R(6) * LBMK_R(0, 2, 2);
  m[19] = R(2) * (LBMK_R(0, 0, 2) - LBMK_R(0, 2, 0)) + R(3) * (LBMK_R(2, 2, 0) - LBMK_R(2, 0, 2));
  m[20] = R(3) * LBMK_R(1, 1, 2) - R(2) * LBMK_R(1, 1, 0);
  m[21] = R(3) * LBMK_R(2, 1, 1) - R(2) * LBMK_R(0, 1, 1);
  m[22] = R(3) * LBMK_R(1, 2, 1) - R(2) * LBMK_R(1, 0, 1);
  m[23] = LBMK_R(1, 2, 0) - LBMK_R(1, 0, 2);
  m[24] = LBMK_R(0, 1, 2) - LBMK_R(2, 1, 0);
  m[25] = LBMK_R(2, 0, 1) - LBMK_R(0, 2, 1);
  m[26] = LBMK_R(1, 1, 1);
}

// r = T^T y: the transpose of moment_forward (T maps raw moments to Eq.
// momentSet moments), over the moments 5..27 only (y[0..3] are ignored).
template <typename R>
__host__ __device__ __forceinline__ void moment_adjoint(const R y[27], R r[27]) {
  const R a16 = R(4) * y[16] - R(8) * y[17];          // common to R000
  const R s2 = y[4] - R(4) * y[16] + R(12) * y[17];   // common to R200, R020, R002
  const R s4 = R(3) * y[16] - R(18) * y[17];          // common to R220, R022, R202
  LBMK_R(0, 0, 0) = a16 - R(2) * y[4];
  LBMK_R(1, 0, 0) = R(4) * (y[13] - y[10]);
  LBMK_R(0, 1, 0) = R(4) * (y[14] - y[11]);
  LBMK_R(0, 0, 1) = R(4) * (y[15] - y[12]);
  LBMK_R(2, 0, 0) = s2 + R(2) * y[5] - R(4) * y[18];
  LBMK_R(0, 2, 0) = s2 - y[5] + y[6] + R(2) * y[18] - R(2) * y[19];
  LBMK_R(0, 0, 2) = s2 - y[5] - y[6] + R(2) * y[18] + R(2) * y[19];
  LBMK_R(1, 1, 0) = y[7] - R(2) * y[20];
  LBMK_R(0, 1, 1) = y[8] - R(2) * y[21];
  LBMK_R(1, 0, 1) = y[9] - R(2) * y[22];
  LBMK_R(1, 2, 0) = R(3) * y[10] - R(6) * y[13] + y[23];
  LBMK_R(1, 0, 2) = R(3) * y[10] - R(6) * y[13] - y[23];
  LBMK_R(0, 1, 2) = R(3) * y[11] - R(6) * y[14] + y[24];
  LBMK_R(2, 1, 0) = R(3) * y[11] - R(6) * y[14] - y[24];
  LBMK_R(2, 0, 1) = R(3) * y[12] - R(6) * y[15] + y[25];
  LBMK_R(0, 2, 1) = R(3) * y[12] - R(6) * y[15] - y[25];
  LBMK_R(1, 2, 2) = R(9) * y[13];
  LBMK_R(2, 1, 2) = R(9) * y[14];
  LBMK_R(2, 2, 1) = R(9) * y[15];
  LBMK_R(2, 2, 0) = s4 + R(3) * y[18] + R(3) * y[19];
  LBMK_R(0, 2, 2) = s4 - R(6) * y[18];
  LBMK_R(2, 0, 2) = s4 + R(3) * y[18] - R(3) * y[19];
  LBMK_R(2, 2, 2) = R(27) * y[17];
  LBMK_R(1, 1, 2) = R(3) * y[20];
  LBMK_R(2, 1, 1) = R(3) * y[21];
  LBMK_R(1, 2, 1) = R(3) * y[22];
  LBMK_R(1, 1, 1) = y[26];
}
#undef LBMK_R

// Full 27x27 transformation matrix as the kernels apply it, column t = tensor
// index (host helper for the self-check; the kernels never form it).
inline void moment_matrix_tensor(double M[27][27]) {
  for (int t = 0; t < Q; ++t) {
    double v[27] = {0};
    v[t] = 1.0;
    raw_forward(v);
    double m[27];
    moment_forward(v, m);
    for (int j = 0; j < Q; ++j) M[j][t] = m[j];
  }
}

// SplitMix64 finaliser (Steele, Lea & Flood, OOPSLA 2014) and the inlet-noise
// variate xi in [-1, 1) keyed by (seed, step, node, component).
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ double inlet_noise(uint64_t seed, int64_t step, int64_t node, int comp) {
  uint64_t h = splitmix64(seed);
  h = splitmix64(h ^ (uint64_t)step);
  h = splitmix64(h ^ (uint64_t)node);
  h = splitmix64(h ^ (uint64_t)comp);
  return (double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

}  // namespace lbmk
