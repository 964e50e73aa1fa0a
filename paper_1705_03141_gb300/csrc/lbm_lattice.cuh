// D3Q27 lattice and moment transforms used by the kernels.
//
// Velocities are held in tensor order t = (cx+1) + 3(cy+1) + 9(cz+1), so the
// rest velocity is t = 13 and the opposite of t is 26 - t.  The D3Q27 weights
// of Sec. II are the products of the D1Q3 weights (1/6, 2/3, 1/6) of the three
// components.  The paper's own direction order (Eq. velSet, fixed by rows 2-4
// of the printed M in App. A) is used only at the C ABI.
//
// Moments.  The raw moments R_abc = sum_i cx^a cy^b cz^c f_i (a,b,c in 0..2)
// follow from three one-dimensional 3-point transforms (one per axis,
// raw_forward; raw_inverse undoes them).  The moments m_1..m_27 of
// Eq. (momentSet) are sparse integer combinations of the R_abc
// (moment_forward, M = T V3), and T has a sparse block inverse
// (moment_inverse_add), so the kernels never hold a dense 27x27 matrix.
#pragma once
#include <stdint.h>

#include <type_traits>

#include "lbm_f2.cuh"

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

// c_T . (a0, a1, a2) with the zero components of c_T left out (IEEE arithmetic
// cannot drop a product with zero on its own).
template <int C, typename R>
__host__ __device__ __forceinline__ R signed_(R a) {
  if constexpr (C > 0) return a;
  else return -a;
}
template <int T, typename R>
__host__ __device__ __forceinline__ R cdot(R a0, R a1, R a2) {
  constexpr int c0 = cx_of(T), c1 = cy_of(T), c2 = cz_of(T);
  if constexpr (c0 != 0 && c1 != 0 && c2 != 0) return signed_<c0>(a0) + signed_<c1>(a1) + signed_<c2>(a2);
  else if constexpr (c0 != 0 && c1 != 0) return signed_<c0>(a0) + signed_<c1>(a1);
  else if constexpr (c0 != 0 && c2 != 0) return signed_<c0>(a0) + signed_<c2>(a2);
  else if constexpr (c1 != 0 && c2 != 0) return signed_<c1>(a1) + signed_<c2>(a2);
  else if constexpr (c0 != 0) return signed_<c0>(a0);
  else if constexpr (c1 != 0) return signed_<c1>(a1);
  else if constexpr (c2 != 0) return signed_<c2>(a2);
  else return R(0);
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
#if defined(__CUDA_ARCH__)
// FP32 on the device: the y and z transforms treat the lines at x-index 0 and 2 alike, so
// those two lines go through one packed FP32x2 transform (a - b as fma(b, -1, a): the
// same rounding as the subtraction); the values and their rounding are the scalar ones.
__device__ __forceinline__ void tri_forward2(float& a0, float& a2, float& b0, float& b2, float& c0, float& c2) {
  const float2 a = make_float2(a0, a2), b = make_float2(b0, b2), c = make_float2(c0, c2);
  const float2 sum = __fadd2_rn(c, a), d = __ffma2_rn(a, make_float2(-1.f, -1.f), c);
  const float2 o = __fadd2_rn(sum, b);
  a0 = o.x;
  a2 = o.y;
  b0 = d.x;
  b2 = d.y;
  c0 = sum.x;
  c2 = sum.y;
}
__device__ __forceinline__ void tri_inverse2(float& a0, float& a2, float& b0, float& b2, float& c0, float& c2) {
  const float2 k0 = make_float2(a0, a2), k1 = make_float2(b0, b2), k2 = make_float2(c0, c2);
  const float2 h2 = __fmul2_rn(make_float2(0.5f, 0.5f), k2);
  const float2 a = __ffma2_rn(make_float2(-0.5f, -0.5f), k1, h2);
  const float2 b = __ffma2_rn(k2, make_float2(-1.f, -1.f), k0);
  const float2 c = __ffma2_rn(make_float2(0.5f, 0.5f), k1, h2);
  a0 = a.x;
  a2 = a.y;
  b0 = b.x;
  b2 = b.y;
  c0 = c.x;
  c2 = c.y;
}
#endif

template <typename R>
__host__ __device__ __forceinline__ void raw_forward(R v[27]) {
#pragma unroll
  for (int l = 0; l < 9; ++l) tri_forward(v[3 * l + 0], v[3 * l + 1], v[3 * l + 2]);  // x
#if defined(__CUDA_ARCH__)
  if constexpr (std::is_same<R, float>::value) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {  // y: lines (x, z) = (0|2, k), then (1, k)
      tri_forward2(v[9 * k], v[9 * k + 2], v[9 * k + 3], v[9 * k + 5], v[9 * k + 6], v[9 * k + 8]);
      tri_forward(v[9 * k + 1], v[9 * k + 4], v[9 * k + 7]);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {  // z: lines (x, y) = (0|2, j), then (1, j)
      tri_forward2(v[3 * j], v[3 * j + 2], v[3 * j + 9], v[3 * j + 11], v[3 * j + 18], v[3 * j + 20]);
      tri_forward(v[3 * j + 1], v[3 * j + 10], v[3 * j + 19]);
    }
    return;
  }
#endif
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    int base = (l % 3) + 9 * (l / 3);
    tri_forward(v[base], v[base + 3], v[base + 6]);  // y
  }
#pragma unroll
  for (int l = 0; l < 9; ++l) tri_forward(v[l], v[l + 9], v[l + 18]);  // z
}

// inverse of tri_forward: (k0, k1, k2) -> ((k2 - k1)/2, k0 - k2, (k2 + k1)/2).
template <typename R>
__host__ __device__ __forceinline__ void tri_inverse(R& a, R& b, R& c) {
  const R k0 = a, k1 = b, k2 = c;
  const R h2 = R(0.5) * k2;
  a = fma_(R(-0.5), k1, h2);
  b = k0 - k2;
  c = fma_(R(0.5), k1, h2);
}

// populations from raw moments: the inverse of raw_forward (z, then y, then x).
template <typename R>
__host__ __device__ __forceinline__ void raw_inverse(R v[27]) {
#if defined(__CUDA_ARCH__)
  if constexpr (std::is_same<R, float>::value) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {  // z
      tri_inverse2(v[3 * j], v[3 * j + 2], v[3 * j + 9], v[3 * j + 11], v[3 * j + 18], v[3 * j + 20]);
      tri_inverse(v[3 * j + 1], v[3 * j + 10], v[3 * j + 19]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {  // y
      tri_inverse2(v[9 * k], v[9 * k + 2], v[9 * k + 3], v[9 * k + 5], v[9 * k + 6], v[9 * k + 8]);
      tri_inverse(v[9 * k + 1], v[9 * k + 4], v[9 * k + 7]);
    }
#pragma unroll
    for (int l = 0; l < 9; ++l) tri_inverse(v[3 * l + 0], v[3 * l + 1], v[3 * l + 2]);  // x
    return;
  }
#endif
#pragma unroll
  for (int l = 0; l < 9; ++l) tri_inverse(v[l], v[l + 9], v[l + 18]);
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    int base = (l % 3) + 9 * (l / 3);
    tri_inverse(v[base], v[base + 3], v[base + 6]);
  }
#pragma unroll
  for (int l = 0; l < 9; ++l) tri_inverse(v[3 * l + 0], v[3 * l + 1], v[3 * l + 2]);
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
  m[4] = fma_(R(-2), LBMK_R(0, 0, 0), S2);                                   // -2<1> + <|c|^2>
  m[5] = fma_(R(3), LBMK_R(2, 0, 0), -S2);                                   // 2<cx^2> - <cy^2+cz^2>
  m[6] = LBMK_R(0, 2, 0) - LBMK_R(0, 0, 2);                                  // <cy^2 - cz^2>
  m[7] = LBMK_R(1, 1, 0);                                                    // <cx cy>
  m[8] = LBMK_R(0, 1, 1);                                                    // <cy cz>
  m[9] = LBMK_R(1, 0, 1);                                                    // <cz cx>
  const R Ax = LBMK_R(1, 2, 0) + LBMK_R(1, 0, 2), Ay = LBMK_R(0, 1, 2) + LBMK_R(2, 1, 0);
  const R Az = LBMK_R(2, 0, 1) + LBMK_R(0, 2, 1);
  m[10] = fma_(R(3), Ax, R(-4) * LBMK_R(1, 0, 0));
  m[11] = fma_(R(3), Ay, R(-4) * LBMK_R(0, 1, 0));
  m[12] = fma_(R(3), Az, R(-4) * LBMK_R(0, 0, 1));
  m[13] = fma_(R(9), LBMK_R(1, 2, 2), fma_(R(-6), Ax, R(4) * LBMK_R(1, 0, 0)));
  m[14] = fma_(R(9), LBMK_R(2, 1, 2), fma_(R(-6), Ay, R(4) * LBMK_R(0, 1, 0)));
  m[15] = fma_(R(9), LBMK_R(2, 2, 1), fma_(R(-6), Az, R(4) * LBMK_R(0, 0, 1)));
  m[16] = fma_(R(3), S4, R(4) * (LBMK_R(0, 0, 0) - S2));                                     // 4<1-|c|^2> + 3<..>
  m[17] = fma_(R(27), LBMK_R(2, 2, 2), fma_(R(-18), S4, fma_(R(12), S2, R(-8) * LBMK_R(0, 0, 0))));
  m[18] = fma_(R(2), LBMK_R(0, 0, 2) + LBMK_R(0, 2, 0),
               fma_(R(3), LBMK_R(2, 2, 0) + LBMK_R(2, 0, 2), fma_(R(-4), LBMK_R(2, 0, 0), R(-6) * LBMK_R(0, 2, 2))));
  m[19] = fma_(R(2), LBMK_R(0, 0, 2) - LBMK_R(0, 2, 0), R(3) * (LBMK_R(2, 2, 0) - LBMK_R(2, 0, 2)));
  m[20] = fma_(R(3), LBMK_R(1, 1, 2), R(-2) * LBMK_R(1, 1, 0));
  m[21] = fma_(R(3), LBMK_R(2, 1, 1), R(-2) * LBMK_R(0, 1, 1));
  m[22] = fma_(R(3), LBMK_R(1, 2, 1), R(-2) * LBMK_R(1, 0, 1));
  m[23] = LBMK_R(1, 2, 0) - LBMK_R(1, 0, 2);
  m[24] = LBMK_R(0, 1, 2) - LBMK_R(2, 1, 0);
  m[25] = LBMK_R(2, 0, 1) - LBMK_R(0, 2, 1);
  m[26] = LBMK_R(1, 1, 1);
}

// r += T^-1 y for a change y of the moments 5..27 (y[0..3] must be zero): the
// inverse of the sparse map of moment_forward, block by block (scalars;
// x-, y-, z-vectors; the three off-diagonal pairs; c_x c_y c_z).
template <typename R>
__host__ __device__ __forceinline__ void moment_inverse_add(const R y[27], R r[27]) {
  // scalar block (moments 1, 5, 6, 7, 17, 18, 19, 20 <-> R000, R200, R020, R002, R220, R202, R022, R222)
  const R dS2 = y[4];                                            // change of R200 + R020 + R002
  const R dS4 = fma_(R(4.0 / 3.0), dS2, R(1.0 / 3.0) * y[16]);    // change of R220 + R202 + R022
  const R d200 = R(1.0 / 3.0) * (y[5] + dS2);
  const R d022 = R(1.0 / 9.0) * fma_(R(2), dS2, fma_(R(-6), d200, fma_(R(3), dS4, -y[18])));
  const R dsum = dS4 - d022;                                      // change of R220 + R202
  const R ddif = R(1.0 / 3.0) * fma_(R(2), y[6], y[19]);          // change of R220 - R202
  const R e = dS2 - d200;
  LBMK_R(2, 0, 0) += d200;
  LBMK_R(0, 2, 0) = fma_(R(0.5), e + y[6], LBMK_R(0, 2, 0));
  LBMK_R(0, 0, 2) = fma_(R(0.5), e - y[6], LBMK_R(0, 0, 2));
  LBMK_R(0, 2, 2) += d022;
  LBMK_R(2, 2, 0) = fma_(R(0.5), dsum + ddif, LBMK_R(2, 2, 0));
  LBMK_R(2, 0, 2) = fma_(R(0.5), dsum - ddif, LBMK_R(2, 0, 2));
  LBMK_R(2, 2, 2) = fma_(R(1.0 / 27.0), fma_(R(-12), dS2, fma_(R(18), dS4, y[17])), LBMK_R(2, 2, 2));
  // vector blocks (moments 2/11/14/24, 3/12/15/25, 4/13/16/26)
  const R vx = R(1.0 / 3.0) * y[10], vy = R(1.0 / 3.0) * y[11], vz = R(1.0 / 3.0) * y[12];
  LBMK_R(1, 2, 0) = fma_(R(0.5), vx + y[23], LBMK_R(1, 2, 0));
  LBMK_R(1, 0, 2) = fma_(R(0.5), vx - y[23], LBMK_R(1, 0, 2));
  LBMK_R(1, 2, 2) = fma_(R(1.0 / 9.0), fma_(R(2), y[10], y[13]), LBMK_R(1, 2, 2));
  LBMK_R(0, 1, 2) = fma_(R(0.5), vy + y[24], LBMK_R(0, 1, 2));
  LBMK_R(2, 1, 0) = fma_(R(0.5), vy - y[24], LBMK_R(2, 1, 0));
  LBMK_R(2, 1, 2) = fma_(R(1.0 / 9.0), fma_(R(2), y[11], y[14]), LBMK_R(2, 1, 2));
  LBMK_R(2, 0, 1) = fma_(R(0.5), vz + y[25], LBMK_R(2, 0, 1));
  LBMK_R(0, 2, 1) = fma_(R(0.5), vz - y[25], LBMK_R(0, 2, 1));
  LBMK_R(2, 2, 1) = fma_(R(1.0 / 9.0), fma_(R(2), y[12], y[15]), LBMK_R(2, 2, 1));
  // off-diagonal pairs (moments 8/21, 9/22, 10/23) and moment 27
  LBMK_R(1, 1, 0) += y[7];
  LBMK_R(1, 1, 2) = fma_(R(1.0 / 3.0), fma_(R(2), y[7], y[20]), LBMK_R(1, 1, 2));
  LBMK_R(0, 1, 1) += y[8];
  LBMK_R(2, 1, 1) = fma_(R(1.0 / 3.0), fma_(R(2), y[8], y[21]), LBMK_R(2, 1, 1));
  LBMK_R(1, 0, 1) += y[9];
  LBMK_R(1, 2, 1) = fma_(R(1.0 / 3.0), fma_(R(2), y[9], y[22]), LBMK_R(1, 2, 1));
  LBMK_R(1, 1, 1) += y[26];
}

// Raw moments of g_i = w_i Q(c_i), Q(c) = C0 + c.V + c.S.c with S symmetric
// (S = {Sxx, Syy, Szz, Sxy, Syz, Sxz}): products of the D1Q3 weight moments
// sum W(c) c^k = 1, 0, 1/3, 0, 1/3 (k = 0..4).  r_abc += sign * R_abc[g] for
// every raw moment except R000 (whose change the caller fixes).
template <typename R>
__host__ __device__ __forceinline__ void closed_raw_add(R r[27], R sign, R C0, const R V[3], const R S[6]) {
  const R t3 = R(1.0 / 3.0) * sign, t9 = R(1.0 / 9.0) * sign, t27 = R(1.0 / 27.0) * sign;
  const R Sxx = S[0], Syy = S[1], Szz = S[2];
  const R a = C0 + Sxx, b = C0 + Syy, c = C0 + Szz, yz = Syy + Szz, xz = Sxx + Szz, xy = Sxx + Syy;
  LBMK_R(1, 0, 0) = fma_(t3, V[0], LBMK_R(1, 0, 0));
  LBMK_R(0, 1, 0) = fma_(t3, V[1], LBMK_R(0, 1, 0));
  LBMK_R(0, 0, 1) = fma_(t3, V[2], LBMK_R(0, 0, 1));
  LBMK_R(2, 0, 0) = fma_(t3, a, fma_(t9, yz, LBMK_R(2, 0, 0)));
  LBMK_R(0, 2, 0) = fma_(t3, b, fma_(t9, xz, LBMK_R(0, 2, 0)));
  LBMK_R(0, 0, 2) = fma_(t3, c, fma_(t9, xy, LBMK_R(0, 0, 2)));
  LBMK_R(2, 2, 0) = fma_(t9, a + Syy, fma_(t27, Szz, LBMK_R(2, 2, 0)));
  LBMK_R(2, 0, 2) = fma_(t9, a + Szz, fma_(t27, Syy, LBMK_R(2, 0, 2)));
  LBMK_R(0, 2, 2) = fma_(t9, b + Szz, fma_(t27, Sxx, LBMK_R(0, 2, 2)));
  LBMK_R(2, 2, 2) = fma_(t27, a + yz, LBMK_R(2, 2, 2));
  const R v0 = t9 * V[0], v1 = t9 * V[1], v2 = t9 * V[2];
  LBMK_R(1, 2, 0) += v0;
  LBMK_R(1, 0, 2) += v0;
  LBMK_R(1, 2, 2) = fma_(t27, V[0], LBMK_R(1, 2, 2));
  LBMK_R(2, 1, 0) += v1;
  LBMK_R(0, 1, 2) += v1;
  LBMK_R(2, 1, 2) = fma_(t27, V[1], LBMK_R(2, 1, 2));
  LBMK_R(2, 0, 1) += v2;
  LBMK_R(0, 2, 1) += v2;
  LBMK_R(2, 2, 1) = fma_(t27, V[2], LBMK_R(2, 2, 1));
  const R u9 = R(2) * t9, u27 = R(2) * t27;
  LBMK_R(1, 1, 0) = fma_(u9, S[3], LBMK_R(1, 1, 0));
  LBMK_R(1, 1, 2) = fma_(u27, S[3], LBMK_R(1, 1, 2));
  LBMK_R(0, 1, 1) = fma_(u9, S[4], LBMK_R(0, 1, 1));
  LBMK_R(2, 1, 1) = fma_(u27, S[4], LBMK_R(2, 1, 1));
  LBMK_R(1, 0, 1) = fma_(u9, S[5], LBMK_R(1, 0, 1));
  LBMK_R(1, 2, 1) = fma_(u27, S[5], LBMK_R(1, 2, 1));
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
