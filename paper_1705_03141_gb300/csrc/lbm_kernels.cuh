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
  double refR[27], refB[27];  // packed storage: rest-state value of each direction in pure red / blue
};

__device__ __forceinline__ bool is_shear_moment(int j) { return j >= 5 && j <= 9; }  // slots s6, s8

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

// ---------------------------------------------------------------------------
// storage policies

template <typename T>
struct PlainStore {  // FP64 or FP32: f^r and f^b planes [2][27][Ns]
  T* A;
  int64_t Ns;
  template <typename R>
  __device__ __forceinline__ void load(int64_t node, int dir, const Phys&, R& fr, R& fb) const {
    fr = (R)__ldcs(A + (int64_t)dir * Ns + node);
    fb = (R)__ldcs(A + (int64_t)(27 + dir) * Ns + node);
  }
  template <typename R>
  __device__ __forceinline__ void store(int64_t node, int dir, const Phys&, R fr, R fb, R) const {
    __stcs(A + (int64_t)dir * Ns + node, (T)fr);
    __stcs(A + (int64_t)(27 + dir) * Ns + node, (T)fb);
  }
};

// Packed 16+16 bit storage: per direction and node one 32-bit word holding
// the total population's deviation from its rest-state value (IEEE half or
// bfloat16, low half) and the red fraction q = f^r/f (unsigned 16-bit fixed
// point, high half, exact 0 and 1).  The rest-state value of direction i is
// q*rho_r0*varphi_i(alpha_r) + (1-q)*rho_b0*w_i, the population of a fluid at
// rest with red fraction q; for i != rest both terms coincide by the density
// ratio relation gamma = (1-alpha_b)/(1-alpha_r) of Sec. II.
template <bool BF16>
struct PackedStore {
  uint32_t* A;
  int64_t Ns;
  __device__ __forceinline__ static float dev_to_float(uint32_t bits) {
    if (BF16) return __bfloat162float(__ushort_as_bfloat16((unsigned short)(bits & 0xFFFFu)));
    return __half2float(__ushort_as_half((unsigned short)(bits & 0xFFFFu)));
  }
  __device__ __forceinline__ static uint32_t float_to_dev(float v) {
    if (BF16) return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
    return (uint32_t)__half_as_ushort(__float2half_rn(v));
  }
  template <typename R>
  __device__ __forceinline__ void load(int64_t node, int dir, const Phys& P, R& fr, R& fb) const {
    const uint32_t w = __ldcs(A + (int64_t)dir * Ns + node);
    const float q = (float)(w >> 16) * (1.0f / 65535.0f);
    const float ref = (float)P.refB[dir] + q * (float)(P.refR[dir] - P.refB[dir]);
    const float f = ref + dev_to_float(w);
    const float r = q * f;
    fr = (R)r;
    fb = (R)(f - r);
  }
  // q_fallback: red fraction used when the total population is too small
  // for f^r/f to mean anything (the node's rho_r/rho).
  template <typename R>
  __device__ __forceinline__ void store(int64_t node, int dir, const Phys& P, R fr, R fb, R q_fallback) const {
    const float f = (float)fr + (float)fb;
    float q = f > 1e-6f ? (float)fr / f : (float)q_fallback;
    q = fminf(fmaxf(q, 0.0f), 1.0f);
    const uint32_t qb = (uint32_t)__float2uint_rn(q * 65535.0f);
    const float qq = (float)qb * (1.0f / 65535.0f);
    const float ref = (float)P.refB[dir] + qq * (float)(P.refR[dir] - P.refB[dir]);
    __stcs(A + (int64_t)dir * Ns + node, (qb << 16) | float_to_dev(f - ref));
  }
};

template <class Store>
struct DensOf { using type = float2; using real = float; };
template <>
struct DensOf<PlainStore<double>> { using type = double2; using real = double; };

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
// load all 27 x 2 populations of a node with the layout of the step about to run
template <class Store, typename R>
__device__ __forceinline__ void load_node(const Store& st, const Phys& P, const NodeMap& nm, int layout,
                                          R fr[27], R fb[27]) {
  if (layout == 0) {
#pragma unroll
    for (int t = 0; t < 27; ++t) st.load(nm.base, t, P, fr[t], fb[t]);
  } else {
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      int64_t node;
      int dir;
      switch (26 - t) {  // read slot S(x, opp(t))
#define LBMK_CASE(k) case k: nm.push<k>(node, dir); break;
        LBMK_CASE(0) LBMK_CASE(1) LBMK_CASE(2) LBMK_CASE(3) LBMK_CASE(4) LBMK_CASE(5) LBMK_CASE(6)
        LBMK_CASE(7) LBMK_CASE(8) LBMK_CASE(9) LBMK_CASE(10) LBMK_CASE(11) LBMK_CASE(12) LBMK_CASE(13)
        LBMK_CASE(14) LBMK_CASE(15) LBMK_CASE(16) LBMK_CASE(17) LBMK_CASE(18) LBMK_CASE(19) LBMK_CASE(20)
        LBMK_CASE(21) LBMK_CASE(22) LBMK_CASE(23) LBMK_CASE(24) LBMK_CASE(25) LBMK_CASE(26)
#undef LBMK_CASE
      }
      st.load(node, dir, P, fr[t], fb[t]);
    }
  }
}

// write the post-collision value of direction t of a node (step parity `odd`)
template <int T, class Store, typename R>
__device__ __forceinline__ void emit(const Store& st, const Phys& P, const NodeMap& nm, bool odd, R fr, R fb, R qf) {
  if (!odd) {
    st.store(nm.base, opp_of(T), P, fr, fb, qf);
  } else {
    int64_t node;
    int dir;
    nm.push<T>(node, dir);
    st.store(node, dir, P, fr, fb, qf);
  }
}

template <int T, class Store, typename R>
struct EmitLoop {
  __device__ __forceinline__ static void run(const Store& st, const Phys& P, const NodeMap& nm, bool odd,
                                             const R* fr, const R* fb, R qf) {
    emit<T>(st, P, nm, odd, fr[T], fb[T], qf);
    EmitLoop<T + 1, Store, R>::run(st, P, nm, odd, fr, fb, qf);
  }
};
template <class Store, typename R>
struct EmitLoop<27, Store, R> {
  __device__ __forceinline__ static void run(const Store&, const Phys&, const NodeMap&, bool, const R*, const R*, R) {}
};

// ---------------------------------------------------------------------------
// body force (Eq. Momentum / Eq. ketFd)
template <typename R>
__device__ __forceinline__ void body_force(const Phys& P, R rho, R F[3]) {
  R k = R(0);
  if (P.force_mode == FORCE_BUOYANCY || P.force_mode == FORCE_DISPERSED) k = rho - (R)P.rho_ref;
  else if (P.force_mode == FORCE_UNIFORM) k = R(1);
  F[0] = k * (R)P.g[0];
  F[1] = k * (R)P.g[1];
  F[2] = k * (R)P.g[2];
}

// Collision of one node, in place: fr/fb (post-streaming, in) become the
// recoloured post-collision values (out).  gphi, grho: isotropic gradients of
// phi and rho.  Returns rho_r/rho in *qf.
//
//   f = f^r + f^b; the operators are linear in the colours, so the MRT step
//   acts on the total f with the total equilibrium
//     f^(e)_i = sum_k rho_k varphi_i^k + rho w_i [3 c.u + 9/2 (c.u)^2 - 3/2 u^2] + Phi_i,
//   Phi_i = 9 w_i nu_bar (c.u)(c.grad rho) (i != rest), -3 nu_bar u.grad rho (rest)
//   (Eq. EES, Eq. varphi_ik, Eq. Phi summed over k; 16/4/1 divided by 48/2 = 9 w_i),
//   and f* = f - M^-1 K M (f - f^(e) + F'/2) + F' + Omega^(2)   (Eq. scoll, Eq. ketF),
//   F'_i = w_i [3 (c - u) + 9 (c.u) c].F (Eq. ketFd),
//   Omega^(2)_i = A |grad phi| [w_i (c.n)^2 - B_i] with B_i = w_i (i != rest),
//   -10/27 (rest) (Eq. perturb with the square, Eq. B_i; A_r = A_b = A),
//   then recolouring: f^r_i = (rho_r/rho) f*_i + beta rho_r rho_b/rho varphi_i(alpha_bar) cos(theta_i).
template <typename R>
__device__ __forceinline__ void collide(const Phys& P, R fr[27], R fb[27], const R gphi[3], const R grho[3], R* qf) {
  R rho_r = R(0), rho_b = R(0);
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    rho_r += fr[t];
    rho_b += fb[t];
  }
  R f[27];
#pragma unroll
  for (int t = 0; t < 27; ++t) f[t] = fr[t] + fb[t];
  const R rho = rho_r + rho_b;
  const R inv_rho = R(1) / rho;
  const R phi = (rho_r - rho_b) * inv_rho;
  R j0 = R(0), j1 = R(0), j2 = R(0);
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    if (cx_of(t) > 0) j0 += f[t];
    if (cx_of(t) < 0) j0 -= f[t];
    if (cy_of(t) > 0) j1 += f[t];
    if (cy_of(t) < 0) j1 -= f[t];
    if (cz_of(t) > 0) j2 += f[t];
    if (cz_of(t) < 0) j2 -= f[t];
  }
  R F[3];
  body_force(P, rho, F);
  const R u0 = (j0 + R(0.5) * F[0]) * inv_rho;
  const R u1 = (j1 + R(0.5) * F[1]) * inv_rho;
  const R u2 = (j2 + R(0.5) * F[2]) * inv_rho;
  const R ar = (R)P.alpha_r, ab = (R)P.alpha_b;
  const R nubar = R(0.5) * ((R(1) + phi) * (R)P.nu_r + (R(1) - phi) * (R)P.nu_b);
  const R s_sh = R(1) / (R(3) * nubar + R(0.5));
  const R prest = R(27.0 / 19.0) * (rho_r * (R(1) - ar) + rho_b * (R(1) - ab));
  const R rest0 = rho_r * ar + rho_b * ab;
  const R uu = u0 * u0 + u1 * u1 + u2 * u2;
  const R uF = u0 * F[0] + u1 * F[1] + u2 * F[2];
  const R ug = u0 * grho[0] + u1 * grho[1] + u2 * grho[2];

  // h = f - f^(e) + F'/2, then its moments
  R h[27];
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    const R w = (R)weight_of(t);
    if (t == REST) {
      const R feq = rest0 - w * R(1.5) * rho * uu - R(3) * nubar * ug;
      h[t] = f[t] - feq - R(1.5) * w * uF;
    } else {
      const R cu = R(cx_of(t)) * u0 + R(cy_of(t)) * u1 + R(cz_of(t)) * u2;
      const R cg = R(cx_of(t)) * grho[0] + R(cy_of(t)) * grho[1] + R(cz_of(t)) * grho[2];
      const R cF = R(cx_of(t)) * F[0] + R(cy_of(t)) * F[1] + R(cz_of(t)) * F[2];
      const R feq = w * (prest + rho * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu) + R(9) * nubar * cu * cg);
      const R fp = w * (R(3) * cF - R(3) * uF + R(9) * cu * cF);
      h[t] = f[t] - feq + R(0.5) * fp;
    }
  }
  raw_forward(h);
  R m[27];
  moment_forward(h, m);
  R y[27];
#pragma unroll
  for (int j = 0; j < 4; ++j) y[j] = R(0);
#pragma unroll
  for (int j = 4; j < 27; ++j) y[j] = -(is_shear_moment(j) ? s_sh * (R)P.invd[j] : (R)P.kd[j]) * m[j];
  R r[27];
  moment_adjoint(y, r);
  raw_adjoint(r);

  // perturbation and recolouring
  const R g2 = gphi[0] * gphi[0] + gphi[1] * gphi[1] + gphi[2] * gphi[2];
  const bool has_n = g2 > R(1e-24);
  const R gn = has_n ? sqrt(g2) : R(0);
  const R inv_gn = has_n ? R(1) / gn : R(0);
  const R n0 = gphi[0] * inv_gn, n1 = gphi[1] * inv_gn, n2 = gphi[2] * inv_gn;
  const R Ag = (R)P.A * gn;
  const R abar = R(0.5) * ((R(1) + phi) * ar + (R(1) - phi) * ab);
  const R rec = (R)P.beta * rho_r * rho_b * inv_rho;
  const R frac = rho_r * inv_rho;
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    const R w = (R)weight_of(t);
    R fstar, rc;
    if (t == REST) {
      fstar = f[t] + r[t] - R(3) * w * uF + Ag * R(10.0 / 27.0);
      rc = R(0);
    } else {
      const R cu = R(cx_of(t)) * u0 + R(cy_of(t)) * u1 + R(cz_of(t)) * u2;
      const R cF = R(cx_of(t)) * F[0] + R(cy_of(t)) * F[1] + R(cz_of(t)) * F[2];
      const R cn = R(cx_of(t)) * n0 + R(cy_of(t)) * n1 + R(cz_of(t)) * n2;
      const R fp = w * (R(3) * cF - R(3) * uF + R(9) * cu * cF);
      fstar = f[t] + r[t] + fp + Ag * w * (cn * cn - R(1));
      const R inv_speed = speed2_of(t) == 1 ? R(1) : (speed2_of(t) == 2 ? R(0.70710678118654752440) : R(0.57735026918962576451));
      rc = rec * R(27.0 / 19.0) * (R(1) - abar) * w * cn * inv_speed;
    }
    const R outr = frac * fstar + rc;
    fr[t] = outr;
    fb[t] = fstar - outr;
  }
  *qf = frac;
}

// Dirichlet inlet node (Sec. IV.A): f^r = f^{r(e)}(rho_r0, u_in, alpha_r) with Phi = 0, f^b = 0.
template <typename R>
__device__ __forceinline__ void inlet_state(const Phys& P, int64_t node_lin, int64_t step, R fr[27], R fb[27]) {
  double u[3] = {0.0, 0.0, P.u_j0};
  if (P.noise_frac != 0.0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] += P.u_j0 * P.noise_frac * inlet_noise(P.seed, step, node_lin, a);
  }
  const R u0 = (R)u[0], u1 = (R)u[1], u2 = (R)u[2];
  const R rho = (R)P.rho_r0, ar = (R)P.alpha_r;
  const R uu = u0 * u0 + u1 * u1 + u2 * u2;
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    const R w = (R)weight_of(t);
    const R cu = R(cx_of(t)) * u0 + R(cy_of(t)) * u1 + R(cz_of(t)) * u2;
    const R vphi = t == REST ? ar : R(27.0 / 19.0) * (R(1) - ar) * w;
    fr[t] = rho * (vphi + w * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu));
    fb[t] = R(0);
  }
}

__device__ __forceinline__ int wrap_or_clamp(int q, int n, int bc_lo, int bc_hi) {
  if (q < 0) return bc_lo == BC_PERIODIC ? q + n : 0;
  if (q >= n) return bc_hi == BC_PERIODIC ? q - n : n - 1;
  return q;
}

// ---------------------------------------------------------------------------
// pass 1: density / phase field
template <class Store>
__global__ void __launch_bounds__(NTHREADS) k_density(Store st, Geom G, Phys P, int layout,
                                                      typename DensOf<Store>::type* __restrict__ dens,
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
  load_node(st, P, nm, layout, fr, fb);
  D rr = D(0), rb = D(0);
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    rr += fr[t];
    rb += fb[t];
  }
  if (is_inlet(G, x, y, z)) {
    rr = (D)P.rho_r0;
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
__global__ void __launch_bounds__(NTHREADS, MINB) k_collide_stream(Store st, const __grid_constant__ Geom G,
                                                                   const __grid_constant__ Phys P, int odd,
                                                                   const typename DensOf<Store>::type* __restrict__ dens,
                                                                   const long long* __restrict__ step_counter) {
  using D = typename DensOf<Store>::real;
  using DT = typename DensOf<Store>::type;
  using R = D;  // compute type: FP64 for FP64 storage, FP32 otherwise
  __shared__ DT tile[TILE];

  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * BZ;
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
  const bool active = x < G.nx && y < G.ny && z < G.nz;

  NodeMap nm;
  R fr[27], fb[27];
  if (active) {
    nm.init(G, x, y, z);
    load_node(st, P, nm, odd, fr, fb);
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

  R qf;
  if (is_inlet(G, x, y, z)) {
    inlet_state(P, dnode(G, x, y, z), (int64_t)*step_counter, fr, fb);
    qf = R(1);
  } else {
    collide(P, fr, fb, gphi, grho, &qf);
  }
  EmitLoop<0, Store, R>::run(st, P, nm, odd != 0, fr, fb, qf);
}

// convective outflow on the z = nz-1 plane (Sec. IV.A), after the step that
// produced time t+1; `layout` is the layout of time t+1.
template <class Store>
__global__ void k_outflow(Store st, Geom G, Phys P, int layout, typename DensOf<Store>::real* __restrict__ top) {
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
  load_node(st, P, below, layout, fr, fb);
  R rho = R(0), mz = R(0);
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    const R v = fr[t] + fb[t];
    rho += v;
    if (cz_of(t) > 0) mz += v;
    if (cz_of(t) < 0) mz -= v;
  }
  R F[3];
  body_force(P, rho, F);
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
    fr[t] = nr;
    fb[t] = nb;
  }
  // write f(N, t+1) where the layout expects it
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    const R sum = fr[t] + fb[t];
    const R qf = sum > R(0) ? fr[t] / sum : R(0.5);
    int64_t node;
    int dir;
    slot_of(here, layout, t, node, dir);
    st.store(node, dir, P, fr[t], fb[t], qf);
  }
}

// ---------------------------------------------------------------------------
// initial state / population I/O / macroscopic fields (FP64 buffers on the device)

// f^k = f^{k(e)}(rho_k, u, alpha_k), Phi = 0; written in layout 0.
template <class Store>
__global__ void k_init(Store st, Geom G, Phys P, const double* __restrict__ rr, const double* __restrict__ rb,
                       const double* __restrict__ u) {
  using R = typename DensOf<Store>::real;
  const int64_t N = (int64_t)G.nx * G.ny * G.nz;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int x = (int)(n % G.nx), y = (int)((n / G.nx) % G.ny), z = (int)(n / ((int64_t)G.nx * G.ny));
  const double u0 = u ? u[n] : 0.0, u1 = u ? u[N + n] : 0.0, u2 = u ? u[2 * N + n] : 0.0;
  const double uu = u0 * u0 + u1 * u1 + u2 * u2;
  const double r = rr[n], b = rb[n];
  const double rho = r + b;
  const int64_t sn = snode(G, x, y, z);
  for (int t = 0; t < 27; ++t) {
    const double w = weight_of(t);
    const double cu = cx_of(t) * u0 + cy_of(t) * u1 + cz_of(t) * u2;
    const double poly = w * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    const double vr = t == REST ? P.alpha_r : 27.0 / 19.0 * (1.0 - P.alpha_r) * w;
    const double vb = t == REST ? P.alpha_b : 27.0 / 19.0 * (1.0 - P.alpha_b) * w;
    const double er = r * (vr + poly), eb = b * (vb + poly);
    st.store(sn, t, P, (R)er, (R)eb, (R)(rho > 0.0 ? r / rho : 0.5));
  }
}

// one direction (paper order pdir) of the canonical [2][27][N] FP64 array <-> storage
template <class Store>
__global__ void k_get_pop(Store st, Geom G, Phys P, int layout, int pdir, double* __restrict__ out_r,
                          double* __restrict__ out_b) {
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
  R fr, fb;
  st.load(node, dir, P, fr, fb);
  out_r[n] = (double)fr;
  out_b[n] = (double)fb;
}

template <class Store>
__global__ void k_set_pop(Store st, Geom G, Phys P, int layout, int pdir, const double* __restrict__ in_r,
                          const double* __restrict__ in_b) {
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
  st.store(node, dir, P, (R)in_r[n], (R)in_b[n], R(0.5));
}

// outflow history := the current populations of the z = nz-1 plane
template <class Store>
__global__ void k_top_from_state(Store st, Geom G, Phys P, int layout, typename DensOf<Store>::real* __restrict__ top) {
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
    st.load(node, dir, P, fr, fb);
    top[(int64_t)t * Pn + pp] = fr;
    top[(int64_t)(27 + t) * Pn + pp] = fb;
  }
}

// rho_r, rho_b, u (Eq. Momentum) into FP64 device buffers (any may be null)
template <class Store>
__global__ void k_macro(Store st, Geom G, Phys P, int layout, double* __restrict__ rr, double* __restrict__ rb,
                        double* __restrict__ u) {
  using R = typename DensOf<Store>::real;
  const int64_t N = (int64_t)G.nx * G.ny * G.nz;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int x = (int)(n % G.nx), y = (int)((n / G.nx) % G.ny), z = (int)(n / ((int64_t)G.nx * G.ny));
  NodeMap nm;
  nm.init(G, x, y, z);
  R fr[27], fb[27];
  load_node(st, P, nm, layout, fr, fb);
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
  double F[3];
  body_force(P, rho, F);
  if (rr) rr[n] = r;
  if (rb) rb[n] = b;
  if (u) {
    u[n] = (j[0] + 0.5 * F[0]) / rho;
    u[N + n] = (j[1] + 0.5 * F[1]) / rho;
    u[2 * N + n] = (j[2] + 0.5 * F[2]) / rho;
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
