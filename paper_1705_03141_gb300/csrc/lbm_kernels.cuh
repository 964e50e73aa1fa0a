// Kernels of the D3Q27 colour-fluid update (templates; instantiated per storage
// type in lbm_kernels_*.cu).
//
// Per time step t (Eq. LBE):
//   pass 1  k_density: rho = rho_r + rho_b and phi = (rho_r - rho_b)/rho
//           (Eq. order) for every node, from the post-streaming populations.
//   pass 2  k_collide_stream: per node, the 26-neighbour isotropic gradients
//           of phi and rho from a shared-memory tile of pass-1 values, then
//           MRT collision with the enhanced equilibrium and MRT forcing,
//           perturbation, recolouring, and streaming in place.
//   bc      k_outflow: convective outflow plane (Sec. IV.A), if present.
//
// In-place streaming (AA pattern).  One population array.  Let S(x, i) be the
// slot (node, direction) where the value leaving node x along c_i arrives:
// x + c_i for interior nodes, wrapped on periodic faces, reflected on
// free-slip faces, bounced back (x, opp(i)) on no-slip faces, and a ghost
// plane z = nz above an outflow face.  S is injective and reversible
// (S(x,i) = (y,j) implies S(y, opp(j)) = (x, opp(i))).
//   even t: node x reads f_i from slot (x, i) and writes f*_i to (x, opp(i));
//   odd t:  node x reads f_i from slot S(x, opp(i)) and writes f*_i to S(x, i).
// Every node reads and writes the same set of slots and no two nodes share a
// slot, so the update is race-free.  After an even step the post-streaming
// value f_i(x) sits in slot S(x, opp(i)) ("layout 1"), after an odd step in
// slot (x, i) ("layout 0").  Layout 0 is also the initial layout.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "lbm_lattice.cuh"

namespace lbmk {

enum { BC_PERIODIC = 0, BC_NOSLIP = 1, BC_FREESLIP = 2, BC_INFLOW_WALL = 3, BC_OUTFLOW = 4 };
enum { FORCE_NONE = 0, FORCE_BUOYANCY = 1, FORCE_DISPERSED = 2, FORCE_UNIFORM = 3 };

constexpr int BX = 32, BY = 4, BZ = 2;  // pass-2 block: one thread per node
constexpr int TX = BX + 2, TY = BY + 2, TZ = BZ + 2;
constexpr int TILE = TX * TY * TZ;
constexpr int NTHREADS = BX * BY * BZ;

struct Geom {
  int nx, ny, nz;
  int64_t Ns;     // slots per direction plane: nx*ny*(nz+2) rounded up (ghost planes z=-1, z=nz)
  int bc[6];
  int inflow;     // inlet disk active on z = 0
  double xc, yc, r2;
};

// Host-side physical parameters (FP64); converted to KConst<R> for the kernels.
struct Phys {
  double rho_r0, rho_b0, alpha_r, alpha_b;
  double nu_r, nu_b, A, beta;
  double kd[27];    // K_j / |M_j|^2 for the moments with fixed rates (0 for j < 4)
  double invd[27];  // 1 / |M_j|^2
  double g[3];
  int force_mode;
  double rho_ref;   // reference density of the force mode
  double u_j0, noise_frac;
  uint64_t seed;
};

// Kernel constants in the compute type R (FP32 kernels read float constants:
// no conversion in the inner loops).
template <typename R>
struct KConst {
  R alpha_r, alpha_b;
  R crest_r, crest_b;      // (27/19)(1 - alpha_k): varphi_i^k = crest_k w_i for moving i
  R nu_mid, nu_half;       // nu_bar = nu_mid + nu_half * phi
  R a_mid, a_half;         // alpha_bar = a_mid + a_half * phi
  R A, beta;
  R kd[27];
  R invd[27];
  R g[3];
  R rho_ref;
  int force_mode;
  // packed storage: rest-state value of a direction of speed class s (|c|^2 = s)
  // at red fraction q is refB[s] + q * dref[s]; dref is zero for moving classes.
  R refB[4], dref[4];
  // inlet (noise in FP64 so that both precisions draw the same variates)
  double rho_r0_d, alpha_r_d, u_j0, noise_frac;
  uint64_t seed;
};

template <typename R>
inline KConst<R> make_kconst(const Phys& P) {
  KConst<R> K;
  K.alpha_r = (R)P.alpha_r;
  K.alpha_b = (R)P.alpha_b;
  K.crest_r = (R)(27.0 / 19.0 * (1.0 - P.alpha_r));
  K.crest_b = (R)(27.0 / 19.0 * (1.0 - P.alpha_b));
  K.nu_mid = (R)(0.5 * (P.nu_r + P.nu_b));
  K.nu_half = (R)(0.5 * (P.nu_r - P.nu_b));
  K.a_mid = (R)(0.5 * (P.alpha_r + P.alpha_b));
  K.a_half = (R)(0.5 * (P.alpha_r - P.alpha_b));
  K.A = (R)P.A;
  K.beta = (R)P.beta;
  for (int j = 0; j < 27; ++j) {
    K.kd[j] = (R)P.kd[j];
    K.invd[j] = (R)P.invd[j];
  }
  for (int a = 0; a < 3; ++a) K.g[a] = (R)P.g[a];
  K.rho_ref = (R)P.rho_ref;
  K.force_mode = P.force_mode;
  const double wcls[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
  for (int s = 0; s < 4; ++s) {
    const double rb = P.rho_b0 * (s == 0 ? P.alpha_b : 27.0 / 19.0 * (1.0 - P.alpha_b) * wcls[s]);
    const double rr = P.rho_r0 * (s == 0 ? P.alpha_r : 27.0 / 19.0 * (1.0 - P.alpha_r) * wcls[s]);
    K.refB[s] = (R)rb;
    K.dref[s] = (R)(s == 0 ? rr - rb : 0.0);  // equal for moving classes (gamma = (1-alpha_b)/(1-alpha_r))
  }
  K.rho_r0_d = P.rho_r0;
  K.alpha_r_d = P.alpha_r;
  K.u_j0 = P.u_j0;
  K.noise_frac = P.noise_frac;
  K.seed = P.seed;
  return K;
}

__host__ __device__ __forceinline__ bool is_shear_moment(int j) { return j >= 5 && j <= 9; }  // slots s6, s8

__host__ __device__ __forceinline__ int64_t snode(const Geom& g, int x, int y, int z) {
  return (int64_t)x + (int64_t)g.nx * ((int64_t)y + (int64_t)g.ny * (int64_t)(z + 1));
}
__host__ __device__ __forceinline__ int64_t dnode(const Geom& g, int x, int y, int z) {
  return (int64_t)x + (int64_t)g.nx * ((int64_t)y + (int64_t)g.ny * (int64_t)z);
}
__device__ __forceinline__ bool is_inlet(const Geom& g, int x, int y, int z) {
  if (!g.inflow || z != 0) return false;
  double dx = x - g.xc, dy = y - g.yc;
  return dx * dx + dy * dy < g.r2;
}

// fast reciprocal / inverse square root: exact in FP64 (oracle parity), MUFU in FP32
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp_(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double sat_(double x) { return fmin(fmax(x, 0.0), 1.0); }
__device__ __forceinline__ float sat_(float x) { return __saturatef(x); }

// Per-node streaming map: for each axis and side the node-index offset of the
// neighbour, whether that side reflects the component (free-slip) and whether
// it bounces back (no-slip).
struct NodeMap {
  int64_t base;
  int off_m[3], off_p[3];
  unsigned flip_m, flip_p, bounce_m, bounce_p;  // bit a per axis

  __device__ __forceinline__ void init(const Geom& g, int x, int y, int z) {
    base = snode(g, x, y, z);
    const int p[3] = {x, y, z};
    const int n[3] = {g.nx, g.ny, g.nz};
    const int stride[3] = {1, g.nx, g.nx * g.ny};
    flip_m = flip_p = bounce_m = bounce_p = 0u;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      off_m[a] = -stride[a];
      off_p[a] = stride[a];
      if (p[a] == 0) {
        const int bc = g.bc[2 * a];
        if (bc == BC_PERIODIC) off_m[a] = (n[a] - 1) * stride[a];
        else if (bc == BC_NOSLIP) bounce_m |= 1u << a;
        else if (bc == BC_FREESLIP || bc == BC_INFLOW_WALL) { off_m[a] = 0; flip_m |= 1u << a; }
      }
      if (p[a] == n[a] - 1) {
        const int bc = g.bc[2 * a + 1];
        if (bc == BC_PERIODIC) off_p[a] = -(n[a] - 1) * stride[a];
        else if (bc == BC_NOSLIP) bounce_p |= 1u << a;
        else if (bc == BC_FREESLIP || bc == BC_INFLOW_WALL) { off_p[a] = 0; flip_p |= 1u << a; }
        // BC_OUTFLOW: off_p stays +stride and lands in the ghost plane z = nz
      }
    }
  }

  // S(x, t): node index and direction of the slot the population leaving along c_t lands in.
  template <int T>
  __device__ __forceinline__ void push(int64_t& node, int& dir) const {
    constexpr int c0 = cx_of(T), c1 = cy_of(T), c2 = cz_of(T);
    bool bounce = false;
    int off = 0, d = T;
    if (c0 < 0) { off += off_m[0]; if (flip_m & 1u) d += 2; bounce |= (bounce_m & 1u) != 0; }
    if (c0 > 0) { off += off_p[0]; if (flip_p & 1u) d -= 2; bounce |= (bounce_p & 1u) != 0; }
    if (c1 < 0) { off += off_m[1]; if (flip_m & 2u) d += 6; bounce |= (bounce_m & 2u) != 0; }
    if (c1 > 0) { off += off_p[1]; if (flip_p & 2u) d -= 6; bounce |= (bounce_p & 2u) != 0; }
    if (c2 < 0) { off += off_m[2]; if (flip_m & 4u) d += 18; bounce |= (bounce_m & 4u) != 0; }
    if (c2 > 0) { off += off_p[2]; if (flip_p & 4u) d -= 18; bounce |= (bounce_p & 4u) != 0; }
    node = bounce ? base : base + off;
    dir = bounce ? opp_of(T) : d;
  }
};

// slot holding the post-streaming population (x, t) in a layout (runtime t)
__device__ __forceinline__ void slot_of(const NodeMap& nm, int layout, int t, int64_t& node, int& dir) {
  if (layout == 0) {
    node = nm.base;
    dir = t;
    return;
  }
  switch (26 - t) {
#define LBMK_CASE(k) case k: nm.push<k>(node, dir); break;
    LBMK_CASE(0) LBMK_CASE(1) LBMK_CASE(2) LBMK_CASE(3) LBMK_CASE(4) LBMK_CASE(5) LBMK_CASE(6)
    LBMK_CASE(7) LBMK_CASE(8) LBMK_CASE(9) LBMK_CASE(10) LBMK_CASE(11) LBMK_CASE(12) LBMK_CASE(13)
    LBMK_CASE(14) LBMK_CASE(15) LBMK_CASE(16) LBMK_CASE(17) LBMK_CASE(18) LBMK_CASE(19) LBMK_CASE(20)
    LBMK_CASE(21) LBMK_CASE(22) LBMK_CASE(23) LBMK_CASE(24) LBMK_CASE(25)
    default: nm.push<26>(node, dir); break;
#undef LBMK_CASE
  }
}

// ---------------------------------------------------------------------------
// storage policies.  `cls` is the speed class |c|^2 of the direction; it is
// unchanged by reflection and bounce-back, so the hot kernels pass it as a
// compile-time value even when the slot's direction index is a runtime value.

template <typename T>
struct PlainStore {  // FP64 or FP32: f^r and f^b planes [2][27][Ns]
  using real = T;
  T* A;
  int64_t Ns;
  template <typename R>
  __device__ __forceinline__ void load(int64_t node, int dir, int, const KConst<R>&, R& fr, R& fb) const {
    fr = (R)__ldcs(A + (int64_t)dir * Ns + node);
    fb = (R)__ldcs(A + (int64_t)(27 + dir) * Ns + node);
  }
  // outr, outb: the two colours; fstar = outr + outb and q = outr / fstar are for packed storage
  template <typename R>
  __device__ __forceinline__ void store(int64_t node, int dir, int, const KConst<R>&, R outr, R outb, R, R) const {
    __stcs(A + (int64_t)dir * Ns + node, (T)outr);
    __stcs(A + (int64_t)(27 + dir) * Ns + node, (T)outb);
  }
};

// Packed 16+16 bit storage: per direction and node one 32-bit word holding
// the total population's deviation from its rest-state value (IEEE half or
// bfloat16, low half) and the red fraction q = f^r/f (unsigned 16-bit fixed
// point, high half, exact 0 and 1).  The rest-state value of a direction is
// q*rho_r0*varphi_i(alpha_r) + (1-q)*rho_b0*w_i, the population of a fluid at
// rest with red fraction q; for moving directions both terms coincide by the
// density ratio relation gamma = (1-alpha_b)/(1-alpha_r) of Sec. II.
template <bool BF16>
struct PackedStore {
  using real = float;
  uint32_t* A;
  int64_t Ns;
  __device__ __forceinline__ static float dev_to_float(uint32_t bits) {
    if (BF16) return __uint_as_float(bits << 16);
    return __half2float(__ushort_as_half((unsigned short)(bits & 0xFFFFu)));
  }
  __device__ __forceinline__ static uint32_t float_to_dev(float v) {
    if (BF16) return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
    return (uint32_t)__half_as_ushort(__float2half_rn(v));
  }
  // 16-bit code k -> k as a float, exactly, through the 2^23 magic number
  __device__ __forceinline__ static float code_to_float(uint32_t k) {
    return __uint_as_float(0x4B000000u | k) - 8388608.0f;
  }
  template <typename R>
  __device__ __forceinline__ void load(int64_t node, int dir, int cls, const KConst<R>& K, R& fr, R& fb) const {
    const uint32_t w = __ldcs(A + (int64_t)dir * Ns + node);
    const float q = code_to_float(w >> 16) * (1.0f / 65535.0f);
    const float f = fmaf(q, (float)K.dref[cls], (float)K.refB[cls]) + dev_to_float(w);
    const float r = q * f;
    fr = (R)r;
    fb = (R)(f - r);
  }
  template <typename R>
  __device__ __forceinline__ void store(int64_t node, int dir, int cls, const KConst<R>& K, R, R, R fstar,
                                        R q) const {
    const float qk = fmaf(__saturatef((float)q), 65535.0f, 8388608.0f);  // rounds to the nearest code
    const uint32_t k = __float_as_uint(qk) & 0xFFFFu;
    const float qq = (qk - 8388608.0f) * (1.0f / 65535.0f);
    const float ref = fmaf(qq, (float)K.dref[cls], (float)K.refB[cls]);
    __stcs(A + (int64_t)dir * Ns + node, (k << 16) | float_to_dev((float)fstar - ref));
  }
};

template <class Store>
struct DensOf { using type = float2; using real = float; };
template <>
struct DensOf<PlainStore<double>> { using type = double2; using real = double; };

// ---------------------------------------------------------------------------
// load all 27 x 2 populations of a node with the layout of the step about to run
template <class Store, typename R>
__device__ __forceinline__ void load_node(const Store& st, const KConst<R>& K, const NodeMap& nm, int layout,
                                          R fr[27], R fb[27]) {
  if (layout == 0) {
#pragma unroll
    for (int t = 0; t < 27; ++t) st.load(nm.base, t, speed2_of(t), K, fr[t], fb[t]);
  } else {
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      int64_t node;
      int dir;
      slot_of(nm, 1, t, node, dir);
      st.load(node, dir, speed2_of(t), K, fr[t], fb[t]);
    }
  }
}

// body force (Eq. Momentum / Eq. ketFd)
template <typename R>
__device__ __forceinline__ void body_force(const KConst<R>& K, R rho, R F[3]) {
  R k = R(0);
  if (K.force_mode == FORCE_BUOYANCY || K.force_mode == FORCE_DISPERSED) k = rho - K.rho_ref;
  else if (K.force_mode == FORCE_UNIFORM) k = R(1);
  F[0] = k * K.g[0];
  F[1] = k * K.g[1];
  F[2] = k * K.g[2];
}

// What the recolouring needs per node after the collision.
template <typename R>
struct Recol {
  R frac;        // rho_r / rho
  R n0, n1, n2;  // unit normal grad(phi)/|grad(phi)| (0 where undefined)
  R rc[4];       // beta rho_r rho_b / rho * varphi_i(alpha_bar) / |c_i| per speed class (rc[0] unused)
  bool has_n;
};

// Collision of one node.  fr/fb: post-streaming populations (in).  On return
// f[t] holds f*_t, the total post-collision population including forcing and
// perturbation, and the returned Recol splits it into colours:
//   f^r_t = frac f*_t + rc[|c_t|^2] (c_t . n),   f^b_t = f*_t - f^r_t.
//
// The operators are linear in the colours, so the MRT step acts on the total f
// (R4).  With the total equilibrium of Eq. (EES) summed over k and the
// forcing of Eq. (ketFd),
//   h_i = f_i - f^(e)_i + F'_i/2 = f_i - w_i Q(c_i) - delta_{i,rest} E,
//   Q(c) = C0 + c.V + c.S.c,   C0 = P - 3/2 rho u^2 + 3/2 u.F,   V = 3 rho u - 3/2 F,
//   S = 9/2 rho u u + 9/2 nu_bar (u g + g u) - 9/4 (u F + F u),
//   E = sum_k rho_k alpha_k - w_rest P - 3 nu_bar u.g,   P = sum_k rho_k crest_k,
// (g = grad rho; Phi_i = 9 w_i nu_bar (c.u)(c.g) for moving i, Eq. Phi with
// 16/4/1 / 48 * 2 = 9 w_i).  The raw moments of w_i c^p are products of the
// D1Q3 weight moments (1, 0, 1/3), so the raw moments of h are those of f
// (one cascade) minus closed forms.  Then f* = f + M^-1(-K M h) + F' + Omega^(2)
// with M^-1 = M^T diag(1/|M_j|^2) (Eq. scoll, Eq. ketF), and
// Omega^(2)_i = A |grad phi| [w_i (c.n)^2 - B_i], B_i = w_i for moving i and
// -10/27 at rest (Eq. perturb with the square, R1; Eq. B_i).
template <typename R>
__device__ __forceinline__ Recol<R> collide(const KConst<R>& K, const R fr[27], const R fb[27], const R gphi[3],
                                            const R grho[3], R f[27]) {
  R rho_r = R(0);
#pragma unroll
  for (int t = 0; t < 27; ++t) rho_r += fr[t];
  R r[27];
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    f[t] = fr[t] + fb[t];
    r[t] = f[t];
  }
  raw_forward(r);
  const R rho = r[0];
  const R rho_b = rho - rho_r;
  const R inv_rho = rcp_(rho);
  R F[3];
  body_force(K, rho, F);
  const R u0 = (r[1] + R(0.5) * F[0]) * inv_rho;
  const R u1 = (r[3] + R(0.5) * F[1]) * inv_rho;
  const R u2 = (r[9] + R(0.5) * F[2]) * inv_rho;
  const R phi = (rho_r - rho_b) * inv_rho;
  const R nubar = K.nu_mid + K.nu_half * phi;
  const R s_sh = rcp_(R(3) * nubar + R(0.5));
  const R Pr = K.crest_r * rho_r + K.crest_b * rho_b;
  const R g0 = grho[0], g1 = grho[1], g2 = grho[2];
  const R uu = u0 * u0 + u1 * u1 + u2 * u2;
  const R uF = u0 * F[0] + u1 * F[1] + u2 * F[2];

  // closed-form raw moments of w_i Q(c_i), subtracted from those of f
  // (delta_rest E only enters R000, which is set to its exact value 0)
  const R C0 = Pr - R(1.5) * rho * uu + R(1.5) * uF;
  const R V0 = R(3) * rho * u0 - R(1.5) * F[0];
  const R V1 = R(3) * rho * u1 - R(1.5) * F[1];
  const R V2 = R(3) * rho * u2 - R(1.5) * F[2];
  const R r45 = R(4.5) * rho, n45 = R(4.5) * nubar;
  const R Sxx = r45 * u0 * u0 + R(2) * n45 * u0 * g0 - R(4.5) * u0 * F[0];
  const R Syy = r45 * u1 * u1 + R(2) * n45 * u1 * g1 - R(4.5) * u1 * F[1];
  const R Szz = r45 * u2 * u2 + R(2) * n45 * u2 * g2 - R(4.5) * u2 * F[2];
  const R Sxy = r45 * u0 * u1 + n45 * (u0 * g1 + u1 * g0) - R(2.25) * (u0 * F[1] + u1 * F[0]);
  const R Syz = r45 * u1 * u2 + n45 * (u1 * g2 + u2 * g1) - R(2.25) * (u1 * F[2] + u2 * F[1]);
  const R Sxz = r45 * u0 * u2 + n45 * (u0 * g2 + u2 * g0) - R(2.25) * (u0 * F[2] + u2 * F[0]);
  const R t3 = R(1.0 / 3.0), t9 = R(1.0 / 9.0), t27 = R(1.0 / 27.0);
#define LBMK_IX(a, b, c) ((a) + 3 * (b) + 9 * (c))
  // mass and momentum of h vanish identically (conserved by the equilibrium with the F/2 shift)
  r[LBMK_IX(0, 0, 0)] = R(0);
  r[LBMK_IX(1, 0, 0)] = R(0);
  r[LBMK_IX(0, 1, 0)] = R(0);
  r[LBMK_IX(0, 0, 1)] = R(0);
  r[LBMK_IX(2, 0, 0)] -= t3 * (C0 + Sxx) + t9 * (Syy + Szz);
  r[LBMK_IX(0, 2, 0)] -= t3 * (C0 + Syy) + t9 * (Sxx + Szz);
  r[LBMK_IX(0, 0, 2)] -= t3 * (C0 + Szz) + t9 * (Sxx + Syy);
  r[LBMK_IX(2, 2, 0)] -= t9 * (C0 + Sxx + Syy) + t27 * Szz;
  r[LBMK_IX(2, 0, 2)] -= t9 * (C0 + Sxx + Szz) + t27 * Syy;
  r[LBMK_IX(0, 2, 2)] -= t9 * (C0 + Syy + Szz) + t27 * Sxx;
  r[LBMK_IX(2, 2, 2)] -= t27 * (C0 + Sxx + Syy + Szz);
  r[LBMK_IX(1, 2, 0)] -= t9 * V0;
  r[LBMK_IX(1, 0, 2)] -= t9 * V0;
  r[LBMK_IX(1, 2, 2)] -= t27 * V0;
  r[LBMK_IX(2, 1, 0)] -= t9 * V1;
  r[LBMK_IX(0, 1, 2)] -= t9 * V1;
  r[LBMK_IX(2, 1, 2)] -= t27 * V1;
  r[LBMK_IX(2, 0, 1)] -= t9 * V2;
  r[LBMK_IX(0, 2, 1)] -= t9 * V2;
  r[LBMK_IX(2, 2, 1)] -= t27 * V2;
  r[LBMK_IX(1, 1, 0)] -= R(2) * t9 * Sxy;
  r[LBMK_IX(1, 1, 2)] -= R(2) * t27 * Sxy;
  r[LBMK_IX(0, 1, 1)] -= R(2) * t9 * Syz;
  r[LBMK_IX(2, 1, 1)] -= R(2) * t27 * Syz;
  r[LBMK_IX(1, 0, 1)] -= R(2) * t9 * Sxz;
  r[LBMK_IX(1, 2, 1)] -= R(2) * t27 * Sxz;
  // R111 of w Q is zero
#undef LBMK_IX

  R m[27];
  moment_forward(r, m);
  R y[27];
#pragma unroll
  for (int j = 0; j < 4; ++j) y[j] = R(0);
#pragma unroll
  for (int j = 4; j < 27; ++j) y[j] = -(is_shear_moment(j) ? s_sh * K.invd[j] : K.kd[j]) * m[j];
  moment_adjoint(y, r);
  raw_adjoint(r);

  // perturbation and recolouring scalars
  Recol<R> out;
  const R G0 = gphi[0], G1 = gphi[1], G2 = gphi[2];
  const R gg = G0 * G0 + G1 * G1 + G2 * G2;
  out.has_n = gg > R(1e-24);
  const R inv_gn = out.has_n ? rsqrt_(gg) : R(0);
  out.n0 = G0 * inv_gn;
  out.n1 = G1 * inv_gn;
  out.n2 = G2 * inv_gn;
  const R Ag = K.A * gg * inv_gn;  // A |grad phi|
  const R abar = K.a_mid + K.a_half * phi;
  const R cr = K.beta * rho_r * rho_b * inv_rho * R(27.0 / 19.0) * (R(1) - abar);
  out.frac = rho_r * inv_rho;
  out.rc[0] = R(0);
  out.rc[1] = cr * R(weight_of(tensor_index(1, 0, 0)));
  out.rc[2] = cr * R(weight_of(tensor_index(1, 1, 0)) * 0.70710678118654752440);
  out.rc[3] = cr * R(weight_of(tensor_index(1, 1, 1)) * 0.57735026918962576451);
  const R Aw1 = Ag * R(weight_of(tensor_index(1, 0, 0)));
  const R Aw2 = Ag * R(weight_of(tensor_index(1, 1, 0)));
  const R Aw3 = Ag * R(weight_of(tensor_index(1, 1, 1)));
  const R uF3 = R(3) * uF;

#pragma unroll
  for (int t = 0; t < 27; ++t) {
    if (t == REST) {
      f[t] = f[t] + r[t] - R(weight_of(REST)) * uF3 + Ag * R(10.0 / 27.0);
    } else {
      const R w = R(weight_of(t));
      const R cu = R(cx_of(t)) * u0 + R(cy_of(t)) * u1 + R(cz_of(t)) * u2;
      const R cF = R(cx_of(t)) * F[0] + R(cy_of(t)) * F[1] + R(cz_of(t)) * F[2];
      const R cn = R(cx_of(t)) * out.n0 + R(cy_of(t)) * out.n1 + R(cz_of(t)) * out.n2;
      const R Aw = speed2_of(t) == 1 ? Aw1 : (speed2_of(t) == 2 ? Aw2 : Aw3);
      const R fp = (R(9) * w * cu) * cF + w * (R(3) * cF - uF3);  // F'_t (Eq. ketFd)
      f[t] = f[t] + r[t] + fp + (Aw * cn * cn - Aw);
    }
  }
  return out;
}

// Dirichlet inlet node (Sec. IV.A): f^r = f^{r(e)}(rho_r0, u_in, alpha_r) with Phi = 0, f^b = 0.
template <typename R>
__device__ __forceinline__ void inlet_state(const KConst<R>& K, int64_t node_lin, int64_t step, R f[27]) {
  double u[3] = {0.0, 0.0, K.u_j0};
  if (K.noise_frac != 0.0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] += K.u_j0 * K.noise_frac * inlet_noise(K.seed, step, node_lin, a);
  }
  const R u0 = (R)u[0], u1 = (R)u[1], u2 = (R)u[2];
  const R rho = (R)K.rho_r0_d, ar = (R)K.alpha_r_d;
  const R uu = u0 * u0 + u1 * u1 + u2 * u2;
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    const R w = (R)weight_of(t);
    const R cu = R(cx_of(t)) * u0 + R(cy_of(t)) * u1 + R(cz_of(t)) * u2;
    const R vphi = t == REST ? ar : R(27.0 / 19.0) * (R(1) - ar) * w;
    f[t] = rho * (vphi + w * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu));
  }
}

__device__ __forceinline__ int wrap_or_clamp(int q, int n, int bc_lo, int bc_hi) {
  if (q < 0) return bc_lo == BC_PERIODIC ? q + n : 0;
  if (q >= n) return bc_hi == BC_PERIODIC ? q - n : n - 1;
  return q;
}

// write direction T of the node (step parity `odd`): colours, f* and red fraction
template <int T, class Store, typename R>
__device__ __forceinline__ void emit(const Store& st, const KConst<R>& K, const NodeMap& nm, bool odd, const R f[27],
                                     const Recol<R>& rc) {
  const R fstar = f[T];
  R outr, q;
  if (T == REST) {
    outr = rc.frac * fstar;
    q = rc.frac;
  } else {
    const R cn = R(cx_of(T)) * rc.n0 + R(cy_of(T)) * rc.n1 + R(cz_of(T)) * rc.n2;
    const R rcol = rc.rc[speed2_of(T)] * cn;
    outr = rc.frac * fstar + rcol;
    q = rc.has_n ? sat_(outr * rcp_(fstar)) : rc.frac;
  }
  const R outb = fstar - outr;
  if (!odd) {
    st.store(nm.base, opp_of(T), speed2_of(T), K, outr, outb, fstar, q);
  } else {
    int64_t node;
    int dir;
    nm.push<T>(node, dir);
    st.store(node, dir, speed2_of(T), K, outr, outb, fstar, q);
  }
}

template <int T, class Store, typename R>
struct EmitLoop {
  __device__ __forceinline__ static void run(const Store& st, const KConst<R>& K, const NodeMap& nm, bool odd,
                                             const R* f, const Recol<R>& rc) {
    emit<T>(st, K, nm, odd, f, rc);
    EmitLoop<T + 1, Store, R>::run(st, K, nm, odd, f, rc);
  }
};
template <class Store, typename R>
struct EmitLoop<27, Store, R> {
  __device__ __forceinline__ static void run(const Store&, const KConst<R>&, const NodeMap&, bool, const R*,
                                             const Recol<R>&) {}
};

// ---------------------------------------------------------------------------
// pass 1: density / phase field
template <class Store>
__global__ void __launch_bounds__(NTHREADS) k_density(Store st, Geom G,
                                                      const __grid_constant__ KConst<typename DensOf<Store>::real> K,
                                                      int layout, typename DensOf<Store>::type* __restrict__ dens,
                                                      int* __restrict__ flag, long long* __restrict__ step_counter) {
  using D = typename DensOf<Store>::real;
  // the counter holds the index of the step being taken (read by pass 2's inlet noise)
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && threadIdx.y == 0 &&
      threadIdx.z == 0)
    *step_counter += 1;
  const int x = blockIdx.x * BX + threadIdx.x;
  const int y = blockIdx.y * BY + threadIdx.y;
  const int z = blockIdx.z * BZ + threadIdx.z;
  if (x >= G.nx || y >= G.ny || z >= G.nz) return;
  NodeMap nm;
  nm.init(G, x, y, z);
  D fr[27], fb[27];
  load_node(st, K, nm, layout, fr, fb);
  D rr = D(0), rb = D(0);
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    rr += fr[t];
    rb += fb[t];
  }
  if (is_inlet(G, x, y, z)) {
    rr = (D)K.rho_r0_d;
    rb = D(0);
  }
  const D rho = rr + rb;
  if (!(rho > D(0)) || !(rho < D(1e30))) atomicOr(flag, 1);
  typename DensOf<Store>::type v;
  v.x = rho;
  v.y = (rr - rb) / rho;
  dens[dnode(G, x, y, z)] = v;
}

// pass 2: gradients + collision + perturbation + recolouring + in-place streaming
template <class Store, int MINB>
__global__ void __launch_bounds__(NTHREADS, MINB)
    k_collide_stream(Store st, const __grid_constant__ Geom G,
                     const __grid_constant__ KConst<typename DensOf<Store>::real> K, int odd,
                     const typename DensOf<Store>::type* __restrict__ dens, const long long* __restrict__ step_counter) {
  using R = typename DensOf<Store>::real;  // compute type: FP64 for FP64 storage, FP32 otherwise
  using DT = typename DensOf<Store>::type;
  __shared__ DT tile[TILE];

  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * BZ;
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
  const bool active = x < G.nx && y < G.ny && z < G.nz;

  NodeMap nm;
  R fr[27], fb[27];
  if (active) {
    nm.init(G, x, y, z);
    load_node(st, K, nm, odd, fr, fb);
  }

  const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
  for (int e = tid; e < TILE; e += NTHREADS) {
    const int tx = e % TX, ty = (e / TX) % TY, tz = e / (TX * TY);
    const int gx = wrap_or_clamp(x0 + tx - 1, G.nx, G.bc[0], G.bc[1]);
    const int gy = wrap_or_clamp(y0 + ty - 1, G.ny, G.bc[2], G.bc[3]);
    const int gz = wrap_or_clamp(z0 + tz - 1, G.nz, G.bc[4], G.bc[5]);
    // out-of-box tail threads of a ragged block read a clamped in-box node
    const int cx = gx < G.nx ? gx : G.nx - 1, cy = gy < G.ny ? gy : G.ny - 1, cz = gz < G.nz ? gz : G.nz - 1;
    tile[e] = dens[dnode(G, cx, cy, cz)];
  }
  __syncthreads();
  if (!active) return;

  R gphi[3] = {R(0), R(0), R(0)}, grho[3] = {R(0), R(0), R(0)};
  const int lx = threadIdx.x + 1, ly = threadIdx.y + 1, lz = threadIdx.z + 1;
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    if (t == REST) continue;
    const DT v = tile[(lx + cx_of(t)) + TX * ((ly + cy_of(t)) + TY * (lz + cz_of(t)))];
    const R w3 = R(3.0 * weight_of(t));
    const R a = w3 * (R)v.y, b = w3 * (R)v.x;
    if (cx_of(t) != 0) { gphi[0] += R(cx_of(t)) * a; grho[0] += R(cx_of(t)) * b; }
    if (cy_of(t) != 0) { gphi[1] += R(cy_of(t)) * a; grho[1] += R(cy_of(t)) * b; }
    if (cz_of(t) != 0) { gphi[2] += R(cz_of(t)) * a; grho[2] += R(cz_of(t)) * b; }
  }

  R f[27];
  Recol<R> rc;
  if (is_inlet(G, x, y, z)) {
    inlet_state(K, dnode(G, x, y, z), (int64_t)*step_counter, f);
    rc.frac = R(1);
    rc.n0 = rc.n1 = rc.n2 = R(0);
    rc.rc[0] = rc.rc[1] = rc.rc[2] = rc.rc[3] = R(0);
    rc.has_n = false;
  } else {
    rc = collide(K, fr, fb, gphi, grho, f);
  }
  EmitLoop<0, Store, R>::run(st, K, nm, odd != 0, f, rc);
}

// write one population pair at (node, dir) of a runtime direction (I/O kernels)
template <class Store, typename R>
__device__ __forceinline__ void store_pair(const Store& st, const KConst<R>& K, int64_t node, int dir, R fr, R fb) {
  const R s = fr + fb;
  const R q = s > R(0) ? fr / s : R(0.5);
  st.store(node, dir, speed2_of(dir), K, fr, fb, s, q);
}

// convective outflow on the z = nz-1 plane (Sec. IV.A), after the step that
// produced time t+1; `layout` is the layout of time t+1.
template <class Store>
__global__ void k_outflow(Store st, Geom G, const __grid_constant__ KConst<typename DensOf<Store>::real> K,
                          int layout, typename DensOf<Store>::real* __restrict__ top) {
  using R = typename DensOf<Store>::real;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= G.nx || y >= G.ny) return;
  const int64_t Pn = (int64_t)G.nx * G.ny;
  const int64_t pp = x + (int64_t)G.nx * y;
  NodeMap below, here;
  below.init(G, x, y, G.nz - 2);
  here.init(G, x, y, G.nz - 1);
  R fr[27], fb[27];
  load_node(st, K, below, layout, fr, fb);
  R rho = R(0), mz = R(0);
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    const R v = fr[t] + fb[t];
    rho += v;
    if (cz_of(t) > 0) mz += v;
    if (cz_of(t) < 0) mz -= v;
  }
  R F[3];
  body_force(K, rho, F);
  const R uz = (mz + R(0.5) * F[2]) / rho;
  const R lam = uz > R(0) ? uz : R(0);
  const R inv = R(1) / (R(1) + lam);
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    R* tr = top + (int64_t)t * Pn + pp;
    R* tb = top + (int64_t)(27 + t) * Pn + pp;
    const R nr = (*tr + lam * fr[t]) * inv;
    const R nb = (*tb + lam * fb[t]) * inv;
    *tr = nr;
    *tb = nb;
    int64_t node;
    int dir;
    slot_of(here, layout, t, node, dir);
    store_pair(st, K, node, dir, nr, nb);
  }
}

// ---------------------------------------------------------------------------
// initial state / population I/O / macroscopic fields (FP64 buffers on the device)

// f^k = f^{k(e)}(rho_k, u, alpha_k), Phi = 0; written in layout 0.
template <class Store>
__global__ void k_init(Store st, Geom G, const __grid_constant__ KConst<typename DensOf<Store>::real> K,
                       const double* __restrict__ rr, const double* __restrict__ rb, const double* __restrict__ u) {
  using R = typename DensOf<Store>::real;
  const int64_t N = (int64_t)G.nx * G.ny * G.nz;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int x = (int)(n % G.nx), y = (int)((n / G.nx) % G.ny), z = (int)(n / ((int64_t)G.nx * G.ny));
  const double u0 = u ? u[n] : 0.0, u1 = u ? u[N + n] : 0.0, u2 = u ? u[2 * N + n] : 0.0;
  const double uu = u0 * u0 + u1 * u1 + u2 * u2;
  const double r = rr[n], b = rb[n];
  const double ar = K.alpha_r_d, ab = 8.0 / 27.0;
  const int64_t sn = snode(G, x, y, z);
  for (int t = 0; t < 27; ++t) {
    const double w = weight_of(t);
    const double cu = cx_of(t) * u0 + cy_of(t) * u1 + cz_of(t) * u2;
    const double poly = w * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    const double vr = t == REST ? ar : 27.0 / 19.0 * (1.0 - ar) * w;
    const double vb = t == REST ? ab : 27.0 / 19.0 * (1.0 - ab) * w;
    store_pair(st, K, sn, t, (R)(r * (vr + poly)), (R)(b * (vb + poly)));
  }
}

// one direction (paper order pdir) of the canonical [2][27][N] FP64 array <-> storage
template <class Store>
__global__ void k_get_pop(Store st, Geom G, const __grid_constant__ KConst<typename DensOf<Store>::real> K,
                          int layout, int pdir, double* __restrict__ out_r, double* __restrict__ out_b) {
  using R = typename DensOf<Store>::real;
  const int64_t N = (int64_t)G.nx * G.ny * G.nz;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int x = (int)(n % G.nx), y = (int)((n / G.nx) % G.ny), z = (int)(n / ((int64_t)G.nx * G.ny));
  NodeMap nm;
  nm.init(G, x, y, z);
  int64_t node;
  int dir;
  const int t = paper_to_tensor(pdir);
  slot_of(nm, layout, t, node, dir);
  R fr, fb;
  st.load(node, dir, speed2_of(t), K, fr, fb);
  out_r[n] = (double)fr;
  out_b[n] = (double)fb;
}

template <class Store>
__global__ void k_set_pop(Store st, Geom G, const __grid_constant__ KConst<typename DensOf<Store>::real> K,
                          int layout, int pdir, const double* __restrict__ in_r, const double* __restrict__ in_b) {
  using R = typename DensOf<Store>::real;
  const int64_t N = (int64_t)G.nx * G.ny * G.nz;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int x = (int)(n % G.nx), y = (int)((n / G.nx) % G.ny), z = (int)(n / ((int64_t)G.nx * G.ny));
  NodeMap nm;
  nm.init(G, x, y, z);
  int64_t node;
  int dir;
  slot_of(nm, layout, paper_to_tensor(pdir), node, dir);
  store_pair(st, K, node, dir, (R)in_r[n], (R)in_b[n]);
}

// outflow history := the current populations of the z = nz-1 plane
template <class Store>
__global__ void k_top_from_state(Store st, Geom G, const __grid_constant__ KConst<typename DensOf<Store>::real> K,
                                 int layout, typename DensOf<Store>::real* __restrict__ top) {
  using R = typename DensOf<Store>::real;
  const int64_t Pn = (int64_t)G.nx * G.ny;
  const int64_t pp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pp >= Pn) return;
  NodeMap nm;
  nm.init(G, (int)(pp % G.nx), (int)(pp / G.nx), G.nz - 1);
  for (int t = 0; t < 27; ++t) {
    int64_t node;
    int dir;
    slot_of(nm, layout, t, node, dir);
    R fr, fb;
    st.load(node, dir, speed2_of(t), K, fr, fb);
    top[(int64_t)t * Pn + pp] = fr;
    top[(int64_t)(27 + t) * Pn + pp] = fb;
  }
}

// rho_r, rho_b, u (Eq. Momentum) into FP64 device buffers (any may be null)
template <class Store>
__global__ void k_macro(Store st, Geom G, const __grid_constant__ KConst<typename DensOf<Store>::real> K, int layout,
                        double* __restrict__ rr, double* __restrict__ rb, double* __restrict__ u) {
  using R = typename DensOf<Store>::real;
  const int64_t N = (int64_t)G.nx * G.ny * G.nz;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int x = (int)(n % G.nx), y = (int)((n / G.nx) % G.ny), z = (int)(n / ((int64_t)G.nx * G.ny));
  NodeMap nm;
  nm.init(G, x, y, z);
  R fr[27], fb[27];
  load_node(st, K, nm, layout, fr, fb);
  double r = 0.0, b = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    r += (double)fr[t];
    b += (double)fb[t];
    const double s = (double)fr[t] + (double)fb[t];
    j[0] += cx_of(t) * s;
    j[1] += cy_of(t) * s;
    j[2] += cz_of(t) * s;
  }
  const double rho = r + b;
  double k = 0.0;
  if (K.force_mode == FORCE_BUOYANCY || K.force_mode == FORCE_DISPERSED) k = rho - (double)K.rho_ref;
  else if (K.force_mode == FORCE_UNIFORM) k = 1.0;
  if (rr) rr[n] = r;
  if (rb) rb[n] = b;
  if (u) {
    u[n] = (j[0] + 0.5 * k * (double)K.g[0]) / rho;
    u[N + n] = (j[1] + 0.5 * k * (double)K.g[1]) / rho;
    u[2 * N + n] = (j[2] + 0.5 * k * (double)K.g[2]) / rho;
  }
}

// ---------------------------------------------------------------------------
// diagnostics: per-block partials (fixed order), then one block combines them.
// partial layout per block: [mass_r, mass_b, p_in, n_in, p_out, n_out, z_le]
constexpr int DIAG_THREADS = 256;
constexpr int DIAG_VALS = 7;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

static __global__ void __launch_bounds__(DIAG_THREADS) k_diag_partial(Geom G, double alpha_r, double alpha_b,
                                                               const double* __restrict__ rr,
                                                               const double* __restrict__ rb,
                                                               double* __restrict__ partial) {
  const int64_t N = (int64_t)G.nx * G.ny * G.nz;
  const int64_t plane = (int64_t)G.nx * G.ny;
  double acc[DIAG_VALS] = {0, 0, 0, 0, 0, 0, -1.0};
  const double cr = 9.0 * (1.0 - alpha_r) / 19.0, cb = 9.0 * (1.0 - alpha_b) / 19.0;
  for (int64_t n = blockIdx.x * (int64_t)DIAG_THREADS + threadIdx.x; n < N; n += (int64_t)gridDim.x * DIAG_THREADS) {
    const double r = rr[n], b = rb[n];
    const double rho = r + b, phi = (r - b) / rho;
    acc[0] += r;
    acc[1] += b;
    const double p = r * cr + b * cb;
    if (phi > 0.99) { acc[2] += p; acc[3] += 1.0; }
    if (phi < -0.99) { acc[4] += p; acc[5] += 1.0; }
    if (phi > 0.0) {
      const int z = (int)(n / plane);
      double cand = (double)z;
      if (z < G.nz - 1) {
        const double r1 = rr[n + plane], b1 = rb[n + plane];
        const double phi1 = (r1 - b1) / (r1 + b1);
        if (phi1 <= 0.0) cand = z + phi / (phi - phi1);
      }
      acc[6] = fmax(acc[6], cand);
    }
  }
  __shared__ double sh[DIAG_VALS][DIAG_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < DIAG_VALS; ++k) {
    const double v = k == 6 ? warp_max(acc[k]) : warp_sum(acc[k]);
    if (lane == 0) sh[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < DIAG_VALS) {
    const int k = threadIdx.x;
    double v = sh[k][0];
    for (int w = 1; w < DIAG_THREADS / 32; ++w) v = k == 6 ? fmax(v, sh[k][w]) : v + sh[k][w];
    partial[(int64_t)blockIdx.x * DIAG_VALS + k] = v;
  }
}

static __global__ void k_diag_final(int nblocks, const double* __restrict__ partial, double* __restrict__ out) {
  // one warp per value, lanes stride over blocks in a fixed order
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= DIAG_VALS) return;
  double v = k == 6 ? -1.0 : 0.0;
  for (int b = lane; b < nblocks; b += 32) {
    const double p = partial[(int64_t)b * DIAG_VALS + k];
    v = k == 6 ? fmax(v, p) : v + p;
  }
  v = k == 6 ? warp_max(v) : warp_sum(v);
  if (lane == 0) out[k] = v;
}

}  // namespace lbmk
