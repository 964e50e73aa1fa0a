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

#include <type_traits>

#include "lbm_lattice.cuh"
#include "lbm_tma.cuh"

namespace lbmk {

enum { BC_PERIODIC = 0, BC_NOSLIP = 1, BC_FREESLIP = 2, BC_INFLOW_WALL = 3, BC_OUTFLOW = 4, BC_HALO = 5 };
enum { FORCE_NONE = 0, FORCE_BUOYANCY = 1, FORCE_DISPERSED = 2, FORCE_UNIFORM = 3 };

constexpr int BX = 32, BY = 4, BZ = 2;  // default block: one thread per node
constexpr int TX = BX + 2, TY = BY + 2, TZ = BZ + 2;
constexpr int TILE = TX * TY * TZ;
constexpr int NTHREADS = BX * BY * BZ;

// Block shapes of the one-node density and collide-stream kernels (256 threads each; a warp is
// always one 32-node x-row): 32 x BY x BZ nodes, and the (rho, phi) halo tile around them.  The
// collide-stream tile is TXT = 36 cells wide (x0-2 .. x0+33; columns 1..34 are read): a tiled
// TMA copy must start on a 16-byte boundary, and x0 - 2 cells of 8 bytes is one.
template <int BY_, int BZ_>
struct Blk {
  static constexpr int BX = 32, BY = BY_, BZ = BZ_;
  static constexpr int TX = BX + 2, TY = BY + 2, TZ = BZ + 2, TILE = TX * TY * TZ;
  static constexpr int TXT = BX + 4, TILET = TXT * TY * TZ;
  static constexpr int NT = BX * BY * BZ, NW = NT / 32;
  static_assert(NT == 256, "256-thread blocks");
};
using BlkDefault = Blk<BY, BZ>;

struct Geom {
  int nx, ny, nz;
  int nxs;        // storage row length: nx rounded up to a multiple of 32 (whole 32-node blocks per row)
  int64_t Ns;     // storage nodes: nxs*ny*(nz+2) rounded up (ghost planes z=-1, z=nz)
  int bc[6];
  int inflow;     // inlet disk active on z = 0
  double xc, yc, r2;
  float* ctop;    // compact storage with an outflow face: the top plane's populations per colour
                  // (the outflow history, authoritative for that plane); null otherwise
};

// Host-side physical parameters (FP64); converted to KConst<R> for the kernels.
struct Phys {
  double rho_r0, rho_b0, alpha_r, alpha_b;
  double nu_r, nu_b, A, beta;
  double rate[27];  // K_j for the moments with fixed rates (0 for j < 4 and the shear slots)
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
  R rate[27];
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
  for (int j = 0; j < 27; ++j) K.rate[j] = (R)P.rate[j];
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
  return (int64_t)x + (int64_t)g.nxs * ((int64_t)y + (int64_t)g.ny * (int64_t)(z + 1));
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
// (the two-lane versions are in lbm_f2.cuh)
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp_(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double sat_(double x) { return fmin(fmax(x, 0.0), 1.0); }
__device__ __forceinline__ float sat_(float x) { return __saturatef(x); }

// ---------------------------------------------------------------------------
// Population storage layout: blocks of 32 consecutive storage nodes; a block
// holds every plane (direction, colour) of its 32 nodes, 32 values per plane.
// A warp's access to one plane is one contiguous 32-value line, and the planes
// of a node sit at compile-time offsets from one per-node address.
__host__ __device__ __forceinline__ int64_t elem_index(int64_t node, int planes, int plane) {
  return ((node >> 5) * planes + plane) * 32 + (node & 31);
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
    const int stride[3] = {1, g.nxs, g.nxs * g.ny};
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
        // BC_OUTFLOW and BC_HALO: off_p stays +stride and lands in the ghost plane z = nz
      }
      // BC_HALO at the low face: off_m stays -stride and lands in the ghost plane z = -1
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

// Streaming map of a node on a "fast row": its y and z neighbours are inside the
// box (a warp is one x-row of a block, so this is warp-uniform) and neither x
// face bounces back.  Storage rows are padded to a multiple of 32 nodes (nxs),
// so a y/z shift moves whole 32-node storage blocks, and S(x, t) only needs the
// element index of plane 0 of the x-shifted node, e[c_x + 1]; a specular
// reflection at an x face turns every direction with that c_x into the one two
// planes away, so it is folded into e as a constant plane shift.  (Lanes past
// nx in the last block of a row are idle; their padding slots are never used.)
struct AoRow {
  int64_t e[3];
  int dxm, dxp;  // e[0] - e[1] and e[2] - e[1]
  // the node's storage block (x >> 5) + (nxs / 32)(y + ny (z + 1)) fits 32 bits; within a block the
  // x neighbours are one element away, across a block edge one block of PLANES planes minus 31
  template <int PLANES>
  __device__ __forceinline__ void init(const Geom& g, int x, int y, int z) {
    const int lane = x & 31;
    const int b = (x >> 5) + (g.nxs >> 5) * (y + g.ny * (z + 1));
    e[1] = (int64_t)b * (PLANES * 32) + lane;
    dxm = lane == 0 ? 31 - 32 * PLANES : -1;
    dxp = lane == 31 ? 32 * PLANES - 31 : 1;
    if (x == 0)
      dxm = g.bc[0] == BC_PERIODIC ? (int)(elem_index(snode(g, g.nx - 1, y, z), PLANES, 0) - e[1]) : 2 * 32;
    if (x == g.nx - 1) dxp = g.bc[1] == BC_PERIODIC ? (int)(elem_index(snode(g, 0, y, z), PLANES, 0) - e[1]) : -2 * 32;
    e[0] = e[1] + dxm;
    e[2] = e[1] + dxp;
  }
  // element offset of the storage row (y + cy, z + cz) from the node's own row (a grid-wide value)
  template <int PLANES>
  __device__ __forceinline__ int row_off(const Geom& g, int cy, int cz) const {
    return cy * (g.nxs * PLANES) + cz * (g.nxs * g.ny * PLANES);
  }
  // element offset of plane 0 of the slot S(x, t) from the node's own plane 0, in 32 bits (a z
  // plane of storage holds fewer than 2^31 elements, checked at creation): slot pointers are the
  // node's base pointer plus one 32-bit offset, one wide multiply-add per access.  nxs is a
  // multiple of 32, so a y step moves nxs / 32 whole blocks of PLANES * 32 elements: nxs * PLANES
  // elements (a z step nxs * ny * PLANES), products the whole grid shares.
  template <int T, int PLANES>
  __device__ __forceinline__ int rel0(const Geom& g) const {
    const int dx = cx_of(T) < 0 ? dxm : (cx_of(T) > 0 ? dxp : 0);
    return dx + cy_of(T) * (g.nxs * PLANES) + cz_of(T) * (g.nxs * g.ny * PLANES);
  }
  // element index of plane 0 of the slot S(x, t) (add the plane of t)
  template <int T, int PLANES>
  __device__ __forceinline__ int64_t slot0(const Geom& g) const {
    return e[cx_of(T) + 1] + (int64_t)(cy_of(T) * (g.nxs * PLANES) + cz_of(T) * (g.nxs * g.ny * PLANES));
  }
};

__device__ __forceinline__ bool fast_row(const Geom& g, int y, int z) {
  return y > 0 && y < g.ny - 1 && z > 0 && z < g.nz - 1 && g.bc[0] != BC_NOSLIP && g.bc[1] != BC_NOSLIP;
}


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

// slot_of for a direction known only at run time (one lane per direction): the slot map of
// NodeMap::push written with selects instead of a switch, so the lanes of a warp do not diverge
__device__ __forceinline__ void slot_of_rt(const NodeMap& nm, int layout, int t, int64_t& node, int& dir) {
  if (layout == 0) {
    node = nm.base;
    dir = t;
    return;
  }
  const int T = 26 - t;  // the slot S(x, opp(t))
  const int c[3] = {cx_of(T), cy_of(T), cz_of(T)};
  int off = 0, d = T;
  bool bounce = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const unsigned bit = 1u << a;
    const int sh = a == 0 ? 2 : (a == 1 ? 6 : 18);
    const bool neg = c[a] < 0, pos = c[a] > 0;
    off += neg ? nm.off_m[a] : (pos ? nm.off_p[a] : 0);
    d += (neg && (nm.flip_m & bit)) ? sh : 0;
    d -= (pos && (nm.flip_p & bit)) ? sh : 0;
    bounce = bounce || (neg && (nm.bounce_m & bit)) || (pos && (nm.bounce_p & bit));
  }
  node = bounce ? nm.base : nm.base + off;
  dir = bounce ? opp_of(T) : d;
}

// ---------------------------------------------------------------------------
// storage policies.  `cls` is the speed class |c|^2 of the direction; it is
// unchanged by reflection and bounce-back, so the hot kernels pass it as a
// compile-time value even when the slot's direction index is a runtime value.

template <typename T>
struct PlainStore {  // FP64 or FP32: f^r and f^b planes [2][27][Ns]
  using real = T;
  static constexpr int PLANES = 54;  // (colour, direction): red 0..26, blue 27..53
  T* A;
  int64_t Ns;
  // loads return the red population and the total f = f^r + f^b
  template <typename R>
  __device__ __forceinline__ void load(int64_t node, int dir, int, const KConst<R>&, R& fr, R& ft) const {
    fr = (R)__ldcs(A + elem_index(node, PLANES, dir));
    ft = fr + (R)__ldcs(A + elem_index(node, PLANES, 27 + dir));
  }
  // accessors by the element index e0 of plane 0 of a node (fast rows)
  template <typename R>
  __device__ __forceinline__ void load_at(int64_t e0, int dir, int, const KConst<R>&, R& fr, R& ft) const {
    fr = (R)__ldcs(A + e0 + dir * 32);
    ft = fr + (R)__ldcs(A + e0 + (27 + dir) * 32);
  }
  // loads that add the red population to acc (red_finish(acc) is the red density)
  template <typename R>
  __device__ __forceinline__ void load_red_at(int64_t e0, int dir, int cls, const KConst<R>& K, R& acc, R& ft) const {
    R fr;
    load_at(e0, dir, cls, K, fr, ft);
    acc += fr;
  }
  template <typename R>
  __device__ __forceinline__ void load_red(int64_t node, int dir, int cls, const KConst<R>& K, R& acc, R& ft) const {
    R fr;
    load(node, dir, cls, K, fr, ft);
    acc += fr;
  }
  template <typename R>
  __device__ __forceinline__ static R red_finish(R acc) { return acc; }
  // by a node's base pointer p1 = A + e1 and a 32-bit element offset (fast rows)
  template <typename R>
  __device__ __forceinline__ void load_red_rel(const T* p1, int rel, int dir, int, const KConst<R>&, R& acc,
                                               R& ft) const {
    const R fr = (R)__ldcs(p1 + (rel + dir * 32));
    ft = fr + (R)__ldcs(p1 + (rel + (27 + dir) * 32));
    acc += fr;
  }
  template <typename R>
  __device__ __forceinline__ void store_rel(T* p1, int rel, int dir, int, const KConst<R>&, R outr, R outb, R,
                                            R) const {
    __stcs(p1 + (rel + dir * 32), (T)outr);
    __stcs(p1 + (rel + (27 + dir) * 32), (T)outb);
  }
  template <typename R>
  __device__ __forceinline__ void store_at(int64_t e0, int dir, int, const KConst<R>&, R outr, R outb, R, R) const {
    __stcs(A + e0 + dir * 32, (T)outr);
    __stcs(A + e0 + (27 + dir) * 32, (T)outb);
  }
  // the two colours as stored (I/O kernels)
  template <typename R>
  __device__ __forceinline__ void load_rb(int64_t node, int dir, int, const KConst<R>&, R& fr, R& fb) const {
    fr = (R)A[elem_index(node, PLANES, dir)];
    fb = (R)A[elem_index(node, PLANES, 27 + dir)];
  }
  // outr, outb: the two colours; fstar = outr + outb and q = outr / fstar are for packed storage
  template <typename R>
  __device__ __forceinline__ void store(int64_t node, int dir, int, const KConst<R>&, R outr, R outb, R, R) const {
    __stcs(A + elem_index(node, PLANES, dir), (T)outr);
    __stcs(A + elem_index(node, PLANES, 27 + dir), (T)outb);
  }
  // two-node accessors (FP32 only): nodes `node` (even) and node+1 of one plane row
  __device__ __forceinline__ void load_s(int64_t node, int dir, float, float, float& fr, float& ft) const {
    fr = (float)__ldcs(A + elem_index(node, PLANES, dir));
    ft = fr + (float)__ldcs(A + elem_index(node, PLANES, 27 + dir));
  }
  __device__ __forceinline__ void store_s(int64_t node, int dir, float, float, float outr, float outb, float,
                                          float) const {
    __stcs(A + elem_index(node, PLANES, dir), (T)outr);
    __stcs(A + elem_index(node, PLANES, 27 + dir), (T)outb);
  }
  __device__ __forceinline__ void load_p(int64_t node, int dir, float, float, F2& fr, F2& ft) const {
    fr = F2(__ldcs(reinterpret_cast<const float2*>(A + elem_index(node, PLANES, dir))));
    ft = fr + F2(__ldcs(reinterpret_cast<const float2*>(A + elem_index(node, PLANES, 27 + dir))));
  }
  __device__ __forceinline__ void store_p(int64_t node, int dir, float, float, F2 outr, F2 outb, F2, F2) const {
    __stcs(reinterpret_cast<float2*>(A + elem_index(node, PLANES, dir)), outr.v);
    __stcs(reinterpret_cast<float2*>(A + elem_index(node, PLANES, 27 + dir)), outb.v);
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
  static constexpr int PLANES = 27;
  static constexpr bool IS_BF16 = BF16;
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
  // word -> (f^r, f); rB, dR: rest-state value of the direction's speed class (dR = 0 for
  // the moving classes, whose rest value does not depend on q: no multiply for them)
  __device__ __forceinline__ static void decode(uint32_t w, float rB, float dR, float& fr, float& f) {
    const float q = code_to_float(w >> 16) * (1.0f / 65535.0f);
    f = (dR != 0.0f ? fmaf(q, dR, rB) : rB) + dev_to_float(w);
    fr = q * f;
  }
  // (f*, q) -> word
  __device__ __forceinline__ static uint32_t encode(float rB, float dR, float fstar, float q) {
    const float qk = fmaf(__saturatef(q), 65535.0f, 8388608.0f);  // rounds to the nearest code
    const uint32_t k = __float_as_uint(qk) & 0xFFFFu;
    const float qq = (qk - 8388608.0f) * (1.0f / 65535.0f);
    return (k << 16) | float_to_dev(fstar - (dR != 0.0f ? fmaf(qq, dR, rB) : rB));
  }
  template <typename R>
  __device__ __forceinline__ void load(int64_t node, int dir, int cls, const KConst<R>& K, R& fr, R& ft) const {
    float a, b;
    decode(__ldcs(A + elem_index(node, PLANES, dir)), (float)K.refB[cls], cls == 0 ? (float)K.dref[0] : 0.0f, a, b);
    fr = (R)a;
    ft = (R)b;
  }
  template <typename R>
  __device__ __forceinline__ void load_at(int64_t e0, int dir, int cls, const KConst<R>& K, R& fr, R& ft) const {
    float a, b;
    decode(__ldcs(A + e0 + dir * 32), (float)K.refB[cls], cls == 0 ? (float)K.dref[0] : 0.0f, a, b);
    fr = (R)a;
    ft = (R)b;
  }
  template <typename R>
  __device__ __forceinline__ void store_at(int64_t e0, int dir, int cls, const KConst<R>& K, R, R, R fstar,
                                           R q) const {
    __stcs(A + e0 + dir * 32, encode((float)K.refB[cls], cls == 0 ? (float)K.dref[0] : 0.0f, (float)fstar, (float)q));
  }
  // loads that add code(q) * f to acc: the red density is (1/65535) sum_i code_i f_i
  // (red_finish), one multiply per node instead of one per direction
  __device__ __forceinline__ static float decode_red(uint32_t w, float rB, float dR, float& acc) {
    const float k = code_to_float(w >> 16);
    const float f = (dR != 0.0f ? fmaf(k * (1.0f / 65535.0f), dR, rB) : rB) + dev_to_float(w);
    acc = fmaf(k, f, acc);
    return f;
  }
  template <typename R>
  __device__ __forceinline__ void load_red_at(int64_t e0, int dir, int cls, const KConst<R>& K, R& acc, R& ft) const {
    float a = (float)acc;
    ft = (R)decode_red(__ldcs(A + e0 + dir * 32), (float)K.refB[cls], cls == 0 ? (float)K.dref[0] : 0.0f, a);
    acc = (R)a;
  }
  template <typename R>
  __device__ __forceinline__ void load_red(int64_t node, int dir, int cls, const KConst<R>& K, R& acc, R& ft) const {
    load_red_at(elem_index(node, PLANES, 0), dir, cls, K, acc, ft);
  }
  template <typename R>
  __device__ __forceinline__ static R red_finish(R acc) { return acc * R(1.0 / 65535.0); }
  // by a node's base pointer p1 = A + e1 and a 32-bit element offset (fast rows)
  template <typename R>
  __device__ __forceinline__ void load_red_rel(const uint32_t* p1, int rel, int dir, int cls, const KConst<R>& K,
                                               R& acc, R& ft) const {
    float a = (float)acc;
    ft = (R)decode_red(__ldcs(p1 + (rel + dir * 32)), (float)K.refB[cls], cls == 0 ? (float)K.dref[0] : 0.0f, a);
    acc = (R)a;
  }
  template <typename R>
  __device__ __forceinline__ void store_rel(uint32_t* p1, int rel, int dir, int cls, const KConst<R>& K, R, R,
                                            R fstar, R q) const {
    __stcs(p1 + (rel + dir * 32), encode((float)K.refB[cls], cls == 0 ? (float)K.dref[0] : 0.0f, (float)fstar,
                                         (float)q));
  }
  template <typename R>
  __device__ __forceinline__ void load_rb(int64_t node, int dir, int cls, const KConst<R>& K, R& fr, R& fb) const {
    R ft;
    load(node, dir, cls, K, fr, ft);
    fb = ft - fr;
  }
  template <typename R>
  __device__ __forceinline__ void store(int64_t node, int dir, int cls, const KConst<R>& K, R, R, R fstar,
                                        R q) const {
    __stcs(A + elem_index(node, PLANES, dir),
           encode((float)K.refB[cls], cls == 0 ? (float)K.dref[0] : 0.0f, (float)fstar, (float)q));
  }
  // two-node accessors: nodes `node` (even) and node+1 of one plane row
  __device__ __forceinline__ void load_s(int64_t node, int dir, float rB, float dR, float& fr, float& ft) const {
    decode(__ldcs(A + elem_index(node, PLANES, dir)), rB, dR, fr, ft);
  }
  __device__ __forceinline__ void store_s(int64_t node, int dir, float rB, float dR, float, float, float fstar,
                                          float q) const {
    __stcs(A + elem_index(node, PLANES, dir), encode(rB, dR, fstar, q));
  }
  __device__ __forceinline__ void load_p(int64_t node, int dir, float rB, float dR, F2& fr, F2& ft) const {
    const uint2 w = __ldcs(reinterpret_cast<const uint2*>(A + elem_index(node, PLANES, dir)));
    decode(w.x, rB, dR, fr.v.x, ft.v.x);
    decode(w.y, rB, dR, fr.v.y, ft.v.y);
  }
  __device__ __forceinline__ void store_p(int64_t node, int dir, float rB, float dR, F2, F2, F2 fstar, F2 q) const {
    __stcs(reinterpret_cast<uint2*>(A + elem_index(node, PLANES, dir)),
           make_uint2(encode(rB, dR, fstar.v.x, q.v.x), encode(rB, dR, fstar.v.y, q.v.y)));
  }
};

template <class Store>
struct DensOf { using type = float2; using real = float; };
template <>
struct DensOf<PlainStore<double>> { using type = double2; using real = double; };

// ---------------------------------------------------------------------------
// load all 27 directions of a node (red and total population) with the layout of the step about to run
template <class Store, typename R>
__device__ __forceinline__ void load_node(const Store& st, const KConst<R>& K, const NodeMap& nm, int layout,
                                          R& rho_r, R ft[27]) {
  R acc = R(0);
  if (layout == 0) {
#pragma unroll
    for (int t = 0; t < 27; ++t) st.load_red(nm.base, t, speed2_of(t), K, acc, ft[t]);
  } else {
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      int64_t node;
      int dir;
      slot_of(nm, 1, t, node, dir);
      st.load_red(node, dir, speed2_of(t), K, acc, ft[t]);
    }
  }
  rho_r += Store::red_finish(acc);
}

// loads of a node on a fast row: even steps read plane t of the node itself,
// odd steps the slot S(x, opp(t))
template <class Store, typename R>
__device__ __forceinline__ void load_node_fast(const Store& st, const KConst<R>& K, const Geom& G, const AoRow& ar,
                                               int odd, R& rho_r, R ft[27]) {
  R acc = R(0);
  const auto* p1 = st.A + ar.e[1];
  if (!odd) {
#pragma unroll
    for (int t = 0; t < 27; ++t) st.load_red_rel(p1, 0, t, speed2_of(t), K, acc, ft[t]);
  } else {
    // slot S(x, opp(t)) is plane T = opp(t) of node x + c_T: the three slots of a row group
    // (c_y, c_z) of T share one row pointer and differ by the x shift dxm / 0 / dxp (t in
    // ascending order, as on even steps)
#pragma unroll
    for (int g9 = 8; g9 >= 0; --g9) {
      const auto* rp = p1 + ar.template row_off<Store::PLANES>(G, g9 % 3 - 1, g9 / 3 - 1);
#pragma unroll
      for (int a = 2; a >= 0; --a) {
        const int T = a + 3 * g9;
        st.load_red_rel(rp, a == 0 ? ar.dxm : (a == 2 ? ar.dxp : 0), T, speed2_of(T), K, acc, ft[26 - T]);
      }
    }
  }
  rho_r += Store::red_finish(acc);
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
  R rho;         // rho of the node (watchdog of the fused density pass)
  R cr;          // beta rho_r rho_b / rho * (27/19)(1 - alpha_bar): rc[s] = cr w_s / |c| (compact record)
  typename MaskOf<R>::type has_n;
};

// Collision of one node.  rho_r: red density (the sum of the red populations, in
// direction order); ft: post-streaming total populations (in).  On return
// f[t] holds f*_t, the total post-collision population including forcing and
// perturbation, and the returned Recol splits it into colours:
//   f^r_t = frac f*_t + rc[|c_t|^2] (c_t . n),   f^b_t = f*_t - f^r_t.
//
// The operators are linear in the colours, so the MRT step acts on the total f
// (R4), and it is carried out on the raw moments R_abc = sum_i cx^a cy^b cz^c f_i:
//   f* = f + M^-1 (-K M h) + F' + Omega^(2),   h = f - f^(e) + F'/2
// (Eq. scoll with Eqs. ketF-ketFd), M = T V3 (V3: raw moments, T: the sparse map
// of Eq. momentSet).  Every term but f has the form w_i Q(c_i) + delta_{i,rest} E
// with Q quadratic in c:
//   f^(e) - F'/2:  C0 = P - 3/2 rho u^2 + 3/2 u.F,  V = 3 rho u - 3/2 F,
//                  S = 9/2 rho u u + 9/2 nu_bar (u g + g u) - 9/4 (u F + F u)
//                  (Eq. EES summed over k, Eq. varphi_ik, Eq. Phi: 16/4/1 / 48 * 2 = 9 w_i),
//   F' + Omega^(2): C0 = -3 u.F - A|grad phi|,  V = 3 F,
//                  S = 9/2 (u F + F u) + A|grad phi| n n
//                  (Eq. ketFd; Eq. perturb with the square, R1, and B_i = w_i for
//                  moving i, -10/27 at rest, Eq. B_i),
// (P = sum_k rho_k crest_k, g = grad rho, n = grad phi/|grad phi|), whose raw
// moments are closed forms; the rest-direction terms only touch R000 (mass),
// which no step changes.  So: R(f) by one cascade, m = T (R(f) - closed) for
// moments 5..27 (mass and momentum of h vanish), R* = R(f) + T^-1(-K m) +
// closed(F' + Omega^(2)), and f* = V3^-1 R* by one inverse cascade.
template <typename R>
__device__ __forceinline__ Recol<R> collide(const KConst<R>& K, const R rho_r, const R ft[27], const R gphi[3],
                                            const R grho[3], R f[27]) {
#pragma unroll
  for (int t = 0; t < 27; ++t) f[t] = ft[t];
  raw_forward(f);  // f holds R(f) from here until raw_inverse
  const R rho = f[0];
  const R rho_b = rho - rho_r;
  const R inv_rho = rcp_(rho);
  R F[3];
  body_force(K, rho, F);
  const R u0 = (f[1] + R(0.5) * F[0]) * inv_rho;
  const R u1 = (f[3] + R(0.5) * F[1]) * inv_rho;
  const R u2 = (f[9] + R(0.5) * F[2]) * inv_rho;
  const R phi = (rho_r - rho_b) * inv_rho;
  const R nubar = K.nu_mid + K.nu_half * phi;
  const R s_sh = rcp_(R(3) * nubar + R(0.5));
  const R Pr = K.crest_r * rho_r + K.crest_b * rho_b;
  const R g0 = grho[0], g1 = grho[1], g2 = grho[2];
  const R uu = u0 * u0 + u1 * u1 + u2 * u2;
  const R uF = u0 * F[0] + u1 * F[1] + u2 * F[2];

  // raw moments of h (mass and momentum of h vanish identically)
  R h[27];
#pragma unroll
  for (int t = 0; t < 27; ++t) h[t] = f[t];
  {
    const R C0 = Pr - R(1.5) * rho * uu + R(1.5) * uF;
    const R V[3] = {R(3) * rho * u0 - R(1.5) * F[0], R(3) * rho * u1 - R(1.5) * F[1], R(3) * rho * u2 - R(1.5) * F[2]};
    const R r45 = R(4.5) * rho, n45 = R(4.5) * nubar;
    const R S[6] = {r45 * u0 * u0 + R(2) * n45 * u0 * g0 - R(4.5) * u0 * F[0],
                    r45 * u1 * u1 + R(2) * n45 * u1 * g1 - R(4.5) * u1 * F[1],
                    r45 * u2 * u2 + R(2) * n45 * u2 * g2 - R(4.5) * u2 * F[2],
                    r45 * u0 * u1 + n45 * (u0 * g1 + u1 * g0) - R(2.25) * (u0 * F[1] + u1 * F[0]),
                    r45 * u1 * u2 + n45 * (u1 * g2 + u2 * g1) - R(2.25) * (u1 * F[2] + u2 * F[1]),
                    r45 * u0 * u2 + n45 * (u0 * g2 + u2 * g0) - R(2.25) * (u0 * F[2] + u2 * F[0])};
    closed_raw_add(h, R(-1), C0, V, S);
  }
  h[0] = R(0);
  h[1] = R(0);
  h[3] = R(0);
  h[9] = R(0);
  R m[27];
  moment_forward(h, m);
#pragma unroll
  for (int j = 0; j < 4; ++j) m[j] = R(0);
#pragma unroll
  for (int j = 4; j < 27; ++j) m[j] = -(is_shear_moment(j) ? s_sh : K.rate[j]) * m[j];  // -K (M h)
  moment_inverse_add(m, f);

  // perturbation and recolouring scalars
  Recol<R> out;
  const R G0 = gphi[0], G1 = gphi[1], G2 = gphi[2];
  const R gg = G0 * G0 + G1 * G1 + G2 * G2;
  out.has_n = gt_(gg, R(1e-24));
  const R inv_gn = select_(out.has_n, rsqrt_(gg), R(0));
  out.n0 = G0 * inv_gn;
  out.n1 = G1 * inv_gn;
  out.n2 = G2 * inv_gn;
  const R Ag = K.A * gg * inv_gn;  // A |grad phi|
  {
    const R V[3] = {R(3) * F[0], R(3) * F[1], R(3) * F[2]};
    const R S[6] = {R(9) * u0 * F[0] + Ag * out.n0 * out.n0, R(9) * u1 * F[1] + Ag * out.n1 * out.n1,
                    R(9) * u2 * F[2] + Ag * out.n2 * out.n2, R(4.5) * (u0 * F[1] + u1 * F[0]) + Ag * out.n0 * out.n1,
                    R(4.5) * (u1 * F[2] + u2 * F[1]) + Ag * out.n1 * out.n2,
                    R(4.5) * (u0 * F[2] + u2 * F[0]) + Ag * out.n0 * out.n2};
    closed_raw_add(f, R(1), R(-3) * uF - Ag, V, S);
  }
  raw_inverse(f);  // f holds f*

  const R abar = K.a_mid + K.a_half * phi;
  const R cr = K.beta * rho_r * rho_b * inv_rho * R(27.0 / 19.0) * (R(1) - abar);
  out.frac = rho_r * inv_rho;
  out.rho = rho;
  out.cr = cr;
  out.rc[0] = R(0);
  out.rc[1] = cr * R(weight_of(tensor_index(1, 0, 0)));
  out.rc[2] = cr * R(weight_of(tensor_index(1, 1, 0)) * 0.70710678118654752440);
  out.rc[3] = cr * R(weight_of(tensor_index(1, 1, 1)) * 0.57735026918962576451);
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
    const R cu = R(cx_of(t)) * u0 + R(cy_of(t)) * u1 + R(cz_of(t)) * u2;  // inlet nodes only
    const R vphi = t == REST ? ar : R(27.0 / 19.0) * (R(1) - ar) * w;
    f[t] = rho * (vphi + w * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu));
  }
}

// coordinate of the (rho, phi) value a tile cell reads along one axis: wrapped on periodic
// faces, the halo plane (-1 or n, filled by the neighbouring slab) on halo faces, else the
// mirror ghost of a wall (the index clamped into the box)
__device__ __forceinline__ int wrap_or_clamp(int q, int n, int bc_lo, int bc_hi) {
  if (q < 0) return bc_lo == BC_PERIODIC ? q + n : (bc_lo == BC_HALO ? -1 : 0);
  if (q >= n) return bc_hi == BC_PERIODIC ? q - n : (bc_hi == BC_HALO ? n : n - 1);
  return q;
}
// the last z plane a tile row may read: nz - 1, or the halo plane nz above a halo face
// (rows past it belong to the ragged tail of the last block and read a clamped row)
__device__ __forceinline__ int tile_zmax(const Geom& G) { return G.bc[5] == BC_HALO ? G.nz : G.nz - 1; }

// ---------------------------------------------------------------------------
// Fused density pass.  The density of node y at t+1 is the sum of the
// populations streamed into it, rho_k(y, t+1) = sum_i f*_i^k(y - c_i, t)
// (boundaries: y is the owner of the slot S(x, i)), so the collide-stream
// kernel of step t can accumulate the next step's (rho, rho_r) while it writes
// f*, and the separate density pass (which rereads every population) is not
// needed.  Accumulators are fixed point, value * 2^22 (resolution 2.4e-7):
// integer addition is exact and associative, so the atomics of different
// blocks give bitwise reproducible sums in any order.  One 64-bit word per node
// holds both, rho_r * 2^54 + rho * 2^22 in two's complement: every partial sum
// is added as one 64-bit integer, and since the total rho * 2^22 lies in
// [0, 2^32) (rho < 1024), the low 32 bits return rho and the high 32 bits
// rho_r (|rho_r| < 512) exactly, whatever the signs of the partial sums.
constexpr float kFixScale = 4194304.0f;
constexpr float kFixInv = 1.0f / 4194304.0f;
__device__ __forceinline__ int to_fix(float v) { return __float2int_rn(v * kFixScale); }
__device__ __forceinline__ unsigned long long pack_fix(float rho, float rho_r) {
  return ((unsigned long long)(unsigned)to_fix(rho_r) << 32) + (unsigned long long)(long long)to_fix(rho);
}

struct FusedIO {
  const unsigned long long* cur;  // fixed-point (rho, rho_r) of the step's input state (index dnode)
  unsigned long long* nxt;        // accumulators of the next state (zero on entry)
  int* flag;                      // watchdog
};

// (rho, phi) of a density-tile cell from the fixed-point accumulators; the
// Dirichlet inlet nodes carry rho_r0 and phi = 1 (as in pass 1)
__device__ __forceinline__ float2 fused_cell(const FusedIO& io, int64_t i) {
  const unsigned long long v = io.cur[i];
  const float rho = (float)(unsigned)v * kFixInv, rr = (float)(int)(unsigned)(v >> 32) * kFixInv;
  return make_float2(rho, __fdividef(rr + rr - rho, rho));
}

// Per-warp rows of next-step densities: warp w (one x-row of the block) owns
// prow[w][K][c] = (rho, rho_r) for its 9 target rows K = (dy+1) + 3(dz+1) and
// the TX columns c = target x - (x0 - 1); columns 0 and TX-1 take what leaves the
// block's x range (the flush maps them through the x faces).  Every entry is
// written once per step, so nothing needs clearing and no atomics are needed.
constexpr int NWARPS = NTHREADS / 32;

// red part of f*_T (the recolouring of emit)
template <int T, bool RECOL, typename R>
__device__ __forceinline__ R red_part(R fstar, const Recol<R>& rc) {
  if (T == REST || !RECOL) return rc.frac * fstar;
  return fma_(rc.rc[speed2_of(T)], cdot<T>(rc.n0, rc.n1, rc.n2), rc.frac * fstar);
}

// Fast rows (a warp is one x-row whose y/z neighbours are inside the box, all
// lanes active): the directions (-1|0|+1, dy, dz) = 3K, 3K+1, 3K+2 of the warp
// all land in the target row (y+dy, z+dz); lane l's target x0+l collects
// z(l) + p(l-1) + m(l+1), summed with two shuffles; lanes 0 and 31 also write
// m(0) / p(31) into the edge columns.
template <int K, bool RECOL, typename R, int BYv = BY, int TXv = TX>
__device__ __forceinline__ void fused_row(float2* prow, const R f[27], const Recol<R>& rc) {
  const int lane = threadIdx.x;
  const float mt = f[3 * K], zt = f[3 * K + 1], pt = f[3 * K + 2];
  const float mr = red_part<3 * K, RECOL>(f[3 * K], rc), zr = red_part<3 * K + 1, RECOL>(f[3 * K + 1], rc),
              pr = red_part<3 * K + 2, RECOL>(f[3 * K + 2], rc);
  const float pt_in = __shfl_up_sync(0xffffffffu, pt, 1), pr_in = __shfl_up_sync(0xffffffffu, pr, 1);
  const float mt_in = __shfl_down_sync(0xffffffffu, mt, 1), mr_in = __shfl_down_sync(0xffffffffu, mr, 1);
  float st = zt, sr = zr;
  if (lane > 0) {
    st += pt_in;
    sr += pr_in;
  }
  if (lane < 31) {
    st += mt_in;
    sr += mr_in;
  }
  float2* row = prow + (((threadIdx.y + BYv * threadIdx.z) * 9 + K) * TXv);
  row[lane + 1] = make_float2(st, sr);
  if (lane == 0) row[0] = make_float2(mt, mr);
  if (lane == 31) row[TXv - 1] = make_float2(pt, pr);
}

// target coordinate along one axis of the slot S(x, t) (c: the component of c_t)
__device__ __forceinline__ void axis_target(int& q, int p, int c, int n, int bc_lo, int bc_hi, bool& bounce,
                                            bool& ghost) {
  if (c == 0) return;
  if (q < 0) {
    if (bc_lo == BC_PERIODIC) q = n - 1;
    else if (bc_lo == BC_NOSLIP) bounce = true;
    else q = p;  // specular reflection keeps the coordinate
  } else if (q >= n) {
    if (bc_hi == BC_PERIODIC) q = 0;
    else if (bc_hi == BC_NOSLIP) bounce = true;
    else if (bc_hi == BC_OUTFLOW) ghost = true;
    else q = p;
  }
}

// Other rows (next to a y or z face, or boxes without fast rows): direction T
// goes straight into the global accumulators of the owner of its slot S(x, T)
// (bounced back to x, reflected, wrapped, or into the ghost plane above an
// outflow face, which no node reads as a density).
template <int T, typename R>
__device__ __forceinline__ void fused_node(const Geom& G, const FusedIO& io, int x, int y, int z, const R f[27],
                                           const Recol<R>& rc) {
  constexpr int dx = cx_of(T), dy = cy_of(T), dz = cz_of(T);
  int tx = x + dx, ty = y + dy, tz = z + dz;
  bool bounce = false, ghost = false;
  axis_target(tx, x, dx, G.nx, G.bc[0], G.bc[1], bounce, ghost);
  axis_target(ty, y, dy, G.ny, G.bc[2], G.bc[3], bounce, ghost);
  axis_target(tz, z, dz, G.nz, G.bc[4], G.bc[5], bounce, ghost);
  if (bounce) {
    tx = x;
    ty = y;
    tz = z;
  } else if (ghost) {
    return;
  }
  atomicAdd(io.nxt + dnode(G, tx, ty, tz), pack_fix((float)f[T], (float)red_part<T, true>(f[T], rc)));
}

// grad phi and grad rho at tile cell (lx, ly, lz) from the (rho, phi) halo tile:
// grad chi = 3 sum_i w_i chi(x + c_i) c_i (the isotropic stencil of Sec. II).
// w_i depends only on the speed class |c_i|^2: the neighbours of one class are
// summed first (signs only), then the class weight multiplies once per component.
template <int CLS, typename R, typename DT, int TXv = TX, int TYv = TY>
__device__ __forceinline__ void class_gradients(const DT* tile, int lx, int ly, int lz, R gphi[3], R grho[3]) {
  R sp[3] = {R(0), R(0), R(0)}, sr[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    if (speed2_of(t) != CLS) continue;
    const DT v = tile[(lx + cx_of(t)) + TXv * ((ly + cy_of(t)) + TYv * (lz + cz_of(t)))];
    if (cx_of(t) > 0) { sp[0] += (R)v.y; sr[0] += (R)v.x; }
    if (cx_of(t) < 0) { sp[0] -= (R)v.y; sr[0] -= (R)v.x; }
    if (cy_of(t) > 0) { sp[1] += (R)v.y; sr[1] += (R)v.x; }
    if (cy_of(t) < 0) { sp[1] -= (R)v.y; sr[1] -= (R)v.x; }
    if (cz_of(t) > 0) { sp[2] += (R)v.y; sr[2] += (R)v.x; }
    if (cz_of(t) < 0) { sp[2] -= (R)v.y; sr[2] -= (R)v.x; }
  }
  const R w = R(3.0 * weight_of(CLS == 1 ? tensor_index(1, 0, 0) : CLS == 2 ? tensor_index(1, 1, 0) : tensor_index(1, 1, 1)));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gphi[k] = fma_(w, sp[k], gphi[k]);
    grho[k] = fma_(w, sr[k], grho[k]);
  }
}
// FP32: a tile cell's (rho, phi) is one register pair, so the two sums of a component advance
// together by one packed FP32x2 add (a fused multiply-add by -1 for a neighbour on the negative
// side, which rounds exactly like the subtraction): the same operations in the same order as
// the scalar sums above, half the instructions.  g[k] = (grad rho, grad phi) along axis k.
template <int CLS, int TXv = TX, int TYv = TY>
__device__ __forceinline__ void class_gradients2(const float2* tile, int lx, int ly, int lz, float2 g[3]) {
  float2 s[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    if (speed2_of(t) != CLS) continue;
    const float2 v = tile[(lx + cx_of(t)) + TXv * ((ly + cy_of(t)) + TYv * (lz + cz_of(t)))];
    if (cx_of(t) > 0) s[0] = __fadd2_rn(s[0], v);
    if (cx_of(t) < 0) s[0] = __ffma2_rn(v, m1, s[0]);
    if (cy_of(t) > 0) s[1] = __fadd2_rn(s[1], v);
    if (cy_of(t) < 0) s[1] = __ffma2_rn(v, m1, s[1]);
    if (cz_of(t) > 0) s[2] = __fadd2_rn(s[2], v);
    if (cz_of(t) < 0) s[2] = __ffma2_rn(v, m1, s[2]);
  }
  const float w = (float)(3.0 * weight_of(CLS == 1 ? tensor_index(1, 0, 0) : CLS == 2 ? tensor_index(1, 1, 0) : tensor_index(1, 1, 1)));
  const float2 w2 = make_float2(w, w);
#pragma unroll
  for (int k = 0; k < 3; ++k) g[k] = __ffma2_rn(w2, s[k], g[k]);
}

template <typename R, typename DT, int TXv = TX, int TYv = TY>
__device__ __forceinline__ void tile_gradients(const DT* tile, int lx, int ly, int lz, R gphi[3], R grho[3]) {
  if constexpr (std::is_same<R, float>::value && std::is_same<DT, float2>::value) {
    float2 g[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    class_gradients2<1, TXv, TYv>(tile, lx, ly, lz, g);
    class_gradients2<2, TXv, TYv>(tile, lx, ly, lz, g);
    class_gradients2<3, TXv, TYv>(tile, lx, ly, lz, g);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      grho[k] = g[k].x;
      gphi[k] = g[k].y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) gphi[k] = grho[k] = R(0);
    class_gradients<1, R, DT, TXv, TYv>(tile, lx, ly, lz, gphi, grho);
    class_gradients<2, R, DT, TXv, TYv>(tile, lx, ly, lz, gphi, grho);
    class_gradients<3, R, DT, TXv, TYv>(tile, lx, ly, lz, gphi, grho);
  }
}

// write direction T of the node (step parity `odd`): colours, f* and red fraction.
// RECOL: some node of the warp has an interface normal (otherwise the
// recolouring term is zero and the red fraction of every direction is rho_r/rho).
// ODDT: the step parity at compile time (0 or 1), or -1 to take it from `odd`
template <int T, bool FAST, bool RECOL, int ODDT, class Store, typename R>
__device__ __forceinline__ void emit(const Store& st, const KConst<R>& K, const Geom& G, const NodeMap& nm,
                                     const AoRow& ar, bool odd_rt, const R f[27], const Recol<R>& rc) {
  const bool odd = ODDT < 0 ? odd_rt : ODDT != 0;
  const R fstar = f[T];
  R outr, q;
  if (T == REST || !RECOL) {
    outr = rc.frac * fstar;
    q = rc.frac;
  } else {
    const R cn = cdot<T>(rc.n0, rc.n1, rc.n2);
    outr = fma_(rc.rc[speed2_of(T)], cn, rc.frac * fstar);
    q = sat_(outr * rcp_(fstar));
  }
  const R outb = fstar - outr;
  if (FAST) {
    auto* p1 = st.A + ar.e[1];
    if (!odd) st.store_rel(p1, 0, opp_of(T), speed2_of(T), K, outr, outb, fstar, q);
    else st.store_rel(p1 + ar.template row_off<Store::PLANES>(G, cy_of(T), cz_of(T)),
                      cx_of(T) < 0 ? ar.dxm : (cx_of(T) > 0 ? ar.dxp : 0), T, speed2_of(T), K, outr, outb, fstar, q);
  } else if (!odd) {
    st.store(nm.base, opp_of(T), speed2_of(T), K, outr, outb, fstar, q);
  } else {
    int64_t node;
    int dir;
    nm.push<T>(node, dir);
    st.store(node, dir, speed2_of(T), K, outr, outb, fstar, q);
  }
}

// FUSED: after each direction (fast rows: each triple of directions), add it to the
// next step's densities (fused density pass; prow, io as in k_collide_stream)
template <int T, class Store, typename R, bool FAST, bool RECOL, bool FUSED, int ODDT = -1, int BYv = BY,
          int TXv = TX>
struct EmitLoop {
  __device__ __forceinline__ static void run(const Store& st, const KConst<R>& K, const Geom& G, const NodeMap& nm,
                                             const AoRow& ar, bool odd, const R* f, const Recol<R>& rc,
                                             float2* prow, const FusedIO& io, int x, int y, int z) {
    emit<T, FAST, RECOL, ODDT>(st, K, G, nm, ar, odd, f, rc);
    if constexpr (FUSED) {
      if constexpr (FAST) {
        if constexpr (T % 3 == 2) fused_row<T / 3, RECOL, R, BYv, TXv>(prow, f, rc);
      } else {
        fused_node<T>(G, io, x, y, z, f, rc);
      }
    }
    EmitLoop<T + 1, Store, R, FAST, RECOL, FUSED, ODDT, BYv, TXv>::run(st, K, G, nm, ar, odd, f, rc, prow, io, x, y, z);
  }
};
template <class Store, typename R, bool FAST, bool RECOL, bool FUSED, int ODDT, int BYv, int TXv>
struct EmitLoop<27, Store, R, FAST, RECOL, FUSED, ODDT, BYv, TXv> {
  __device__ __forceinline__ static void run(const Store&, const KConst<R>&, const Geom&, const NodeMap&,
                                             const AoRow&, bool, const R*, const Recol<R>&, float2*, const FusedIO&,
                                             int, int, int) {}
};

// ---------------------------------------------------------------------------
// pass 1: density / phase field.  FIX: write the fixed-point accumulators of
// the fused density pass instead (priming the fused pass from a stored state).
// write one population pair at (node, dir) of a runtime direction (I/O kernels)
template <class Store, typename R>
__device__ __forceinline__ void store_pair(const Store& st, const KConst<R>& K, int64_t node, int dir, R fr, R fb) {
  const R s = fr + fb;
  const R q = s > R(0) ? fr / s : R(0.5);
  st.store(node, dir, speed2_of(dir), K, fr, fb, s, q);
}

// the sum a warp_allsum over lanes 0..31 gives, with v[l] the value of lane l (the same
// additions in the same order: at each stage lane l adds the value of lane l ^ o); v is consumed
template <typename R>
__device__ __forceinline__ R xor_tree_sum(R v[32]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int l = 0; l < o; ++l) v[l] = v[l] + v[l + o];
  }
  return v[0];
}

// The convective outflow of the step before (Sec. IV.A) for the column (x, y), by one thread:
// the same arithmetic, in the same order, as k_outflow (which gives it to 27 lanes); `layout`
// is the layout of the state the outflow completes.
template <class Store, typename R>
__device__ __forceinline__ void outflow_column(const Store& st, const Geom& G, const KConst<R>& K, int layout, int x,
                                               int y, R* __restrict__ top) {
  NodeMap below, here;
  below.init(G, x, y, G.nz - 2);
  here.init(G, x, y, G.nz - 1);
  R fr[27], fb[27], a[32], m[32];
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    int64_t node;
    int dir;
    slot_of(below, layout, t, node, dir);
    st.load_rb(node, dir, speed2_of(t), K, fr[t], fb[t]);
    const R v = fr[t] + fb[t];
    a[t] = v;
    m[t] = cz_of(t) > 0 ? v : cz_of(t) < 0 ? -v : R(0);
  }
#pragma unroll
  for (int t = 27; t < 32; ++t) a[t] = m[t] = R(0);
  const R rho = xor_tree_sum(a);
  const R mz = xor_tree_sum(m);
  R F[3];
  body_force(K, rho, F);
  const R uz = (mz + R(0.5) * F[2]) / rho;
  const R lam = uz > R(0) ? uz : R(0);
  const R inv = R(1) / (R(1) + lam);
  R* tr = top + ((int64_t)x + (int64_t)G.nx * y) * 64;
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    const R nr = (tr[t] + lam * fr[t]) * inv;
    const R nb = (tr[32 + t] + lam * fb[t]) * inv;
    tr[t] = nr;
    tr[32 + t] = nb;
    int64_t node;
    int dir;
    slot_of(here, layout, t, node, dir);
    store_pair(st, K, node, dir, nr, nb);
  }
}

// top != null (an outflow face): the threads of the plane z = nz-1 first complete the step
// before with its convective outflow (outflow_column), so that k_outflow need not run between
// the steps of a run; the blocks of the top planes start first (z blocks in reverse order).
// Four blocks per SM (64 registers): the outflow path of the top plane may spill, the pass over
// the rest of the box keeps its occupancy (a streaming pass, bound by memory parallelism).
template <class Store, bool FIX, class B = BlkDefault>
__global__ void __launch_bounds__(B::NT, 4) k_density(Store st, Geom G,
                                                      const __grid_constant__ KConst<typename DensOf<Store>::real> K,
                                                      int layout, typename DensOf<Store>::type* __restrict__ dens,
                                                      int* __restrict__ flag,
                                                      unsigned long long* __restrict__ fix,
                                                      typename DensOf<Store>::real* __restrict__ top) {
  using D = typename DensOf<Store>::real;
  const int x = blockIdx.x * B::BX + threadIdx.x;
  const int y = blockIdx.y * B::BY + threadIdx.y;
  const int z = (gridDim.z - 1 - blockIdx.z) * B::BZ + threadIdx.z;
  if (x >= G.nx || y >= G.ny || z >= G.nz) return;
  if (top != nullptr && z == G.nz - 1) outflow_column(st, G, K, layout, x, y, top);
  D rr = D(0), ft[27];
  if (fast_row(G, y, z)) {
    AoRow ar;
    ar.init<Store::PLANES>(G, x, y, z);
    load_node_fast(st, K, G, ar, layout, rr, ft);
  } else {
    NodeMap nm;
    nm.init(G, x, y, z);
    load_node(st, K, nm, layout, rr, ft);
  }
  D rt = D(0);
#pragma unroll
  for (int t = 0; t < 27; ++t) rt += ft[t];
  if (!(rt > D(0)) || !(rt < D(1e30))) atomicOr(flag, 1);
  if constexpr (FIX) {
    fix[dnode(G, x, y, z)] = pack_fix((float)rt, (float)rr);
  } else {
    D rb = rt - rr;
    if (is_inlet(G, x, y, z)) {
      rr = (D)K.rho_r0_d;
      rb = D(0);
    }
    const D rho = rr + rb;
    typename DensOf<Store>::type v;
    v.x = rho;
    v.y = (rr - rb) / rho;
    dens[dnode(G, x, y, z)] = v;
  }
}

// The (rho, phi) halo tile of a collide-stream block through one tiled TMA copy.  The copy cannot
// wrap around a periodic face, so blocks whose tile crosses one fill it with loads instead.
template <class B>
__device__ __forceinline__ bool tile_wraps(const Geom& G, int x0, int y0, int z0) {
  return (x0 == 0 && G.bc[0] == BC_PERIODIC) || (x0 + B::BX >= G.nx && G.bc[1] == BC_PERIODIC) ||
         (y0 == 0 && G.bc[2] == BC_PERIODIC) || (y0 + B::BY >= G.ny && G.bc[3] == BC_PERIODIC) ||
         (z0 == 0 && G.bc[4] == BC_PERIODIC) || (z0 + B::BZ >= G.nz && G.bc[5] == BC_PERIODIC);
}

// In-box ranges of a TMA-copied tile (tile coordinates: column c is x = x0 - 2 + c, row r is
// y = y0 - 1 + r, plane p is z = z0 - 1 + p).  Along z the box reaches the halo planes z = -1 and
// z = nz on halo faces (the tensor covers both ghost planes); every other cell outside these ranges
// is a mirror ghost of a wall, the inlet or the outflow plane: the in-box cell with its coordinates
// clamped, as the loads of wrap_or_clamp give it.
struct TileRange {
  int cx0, cx1, cy0, cy1, cz0, cz1;
  template <class B>
  __device__ __forceinline__ void init(const Geom& G, int x0, int y0, int z0) {
    const int zlo = G.bc[4] == BC_HALO ? -1 : 0, zhi = tile_zmax(G);
    cx0 = max(2 - x0, 0);
    cx1 = min(G.nx + 1 - x0, B::TXT - 1);
    cy0 = max(1 - y0, 0);
    cy1 = min(G.ny - y0, B::TY - 1);
    cz0 = max(zlo + 1 - z0, 0);
    cz1 = min(zhi + 1 - z0, B::TZ - 1);
  }
  template <class B>
  __device__ __forceinline__ bool clamps() const {
    return cx0 > 0 || cx1 < B::TXT - 1 || cy0 > 0 || cy1 < B::TY - 1 || cz0 > 0 || cz1 < B::TZ - 1;
  }
  template <class B>
  __device__ __forceinline__ int src(int c, int r, int p) const {
    return min(max(c, cx0), cx1) + B::TXT * (min(max(r, cy0), cy1) + B::TY * min(max(p, cz0), cz1));
  }
};

// Replace the out-of-box cells of the tile by their clamped in-box cells: the out-of-box columns,
// rows and planes in turn, each cell from the cell with all three coordinates clamped (never an
// out-of-box cell itself, so the three loops need no ordering; corners are written twice with the
// same value).
template <class B, typename DT>
__device__ __forceinline__ void tile_clamp_fix(DT* tile, const TileRange& tr, int tid) {
  const int ncx = tr.cx0 + (B::TXT - 1 - tr.cx1), ncy = tr.cy0 + (B::TY - 1 - tr.cy1),
            ncz = tr.cz0 + (B::TZ - 1 - tr.cz1);
  for (int k = tid; k < ncx * B::TY * B::TZ; k += B::NT) {
    const int j = k % ncx, rp = k / ncx;
    const int c = j < tr.cx0 ? j : tr.cx1 + 1 + (j - tr.cx0), r = rp % B::TY, p = rp / B::TY;
    tile[c + B::TXT * (r + B::TY * p)] = tile[tr.src<B>(c, r, p)];
  }
  for (int k = tid; k < ncy * B::TXT * B::TZ; k += B::NT) {
    const int c = k % B::TXT, jp = k / B::TXT, j = jp % ncy, p = jp / ncy;
    const int r = j < tr.cy0 ? j : tr.cy1 + 1 + (j - tr.cy0);
    tile[c + B::TXT * (r + B::TY * p)] = tile[tr.src<B>(c, r, p)];
  }
  for (int k = tid; k < ncz * B::TXT * B::TY; k += B::NT) {
    const int c = k % B::TXT, jr = k / B::TXT, r = jr % B::TY, j = jr / B::TY;
    const int p = j < tr.cz0 ? j : tr.cz1 + 1 + (j - tr.cz0);
    tile[c + B::TXT * (r + B::TY * p)] = tile[tr.src<B>(c, r, p)];
  }
}

// pass 2: gradients + collision + perturbation + recolouring + in-place streaming.
// counter[t & 1] holds the index t of the step (read by the inlet noise); the
// kernel writes t + 1 into counter[(t + 1) & 1] for the next step, so a
// captured graph of steps needs no parameter updates.  FUSED: (rho, phi) come
// from the fixed-point accumulators of the previous step, and the kernel
// accumulates those of the next step (fused_row, fused_node).
// Split of the tile grid into interior tiles (every row a fast row: 1 <= y, y + BY - 1 <= ny - 2,
// and the same along z) and the boundary tiles around them.
struct TileSplit {
  int ntx, nty, ntz;  // tiles along x, y, z
  int tyb, tzb;       // interior tile rows ty = 1 .. tyb, planes tz = 1 .. tzb
  __host__ __device__ int ny_in() const { return tyb >= 1 ? tyb : 0; }
  __host__ __device__ int nz_in() const { return tzb >= 1 ? tzb : 0; }
  __host__ __device__ int interior() const { return ntx * ny_in() * nz_in(); }
  __host__ __device__ int boundary() const { return ntx * nty * ntz - interior(); }
  // boundary tile b -> tile origin: the tile planes below and above the interior, then the
  // tile rows beside it (x fastest)
  __device__ __forceinline__ void boundary_tile(int b, int BYv, int BZv, int& x0, int& y0, int& z0) const {
    const int xi = b % ntx;
    int p = b / ntx, ty, tz;
    const int nlow = nty, nhigh = (ntz - 1 - nz_in()) * nty;
    if (p < nlow) {
      tz = 0;
      ty = p;
    } else if (p - nlow < nhigh) {
      p -= nlow;
      tz = nz_in() + 1 + p / nty;
      ty = p % nty;
    } else {
      p -= nlow + nhigh;
      const int per = nty - ny_in();  // tile rows beside the interior: 0 and ny_in + 1 ..
      tz = 1 + p / per;
      const int r = p % per;
      ty = r == 0 ? 0 : ny_in() + r;
    }
    x0 = xi * 32;
    y0 = ty * BYv;
    z0 = tz * BZv;
  }
  __device__ __forceinline__ void interior_tile(int i, int BYv, int BZv, int& x0, int& y0, int& z0) const {
    const int xi = i % ntx, p = i / ntx;
    x0 = xi * 32;
    y0 = (1 + p % ny_in()) * BYv;
    z0 = (1 + p / ny_in()) * BZv;
  }
};

// the tile split of the default 32 x BY x BZ blocks, and whether the TMA-pipelined kernel
// (variant 5) takes the interior tiles: reflecting x faces (the staged rows mirror there),
// even nx (8-byte density cells in 16-byte rows) and at least one interior tile
inline TileSplit default_tile_split(const Geom& G) {
  TileSplit ts;
  ts.ntx = (G.nx + 31) / 32;
  ts.nty = (G.ny + BY - 1) / BY;
  ts.ntz = (G.nz + BZ - 1) / BZ;
  ts.tyb = G.ny - 1 - BY >= 0 ? (G.ny - 1 - BY) / BY : 0;
  ts.tzb = G.nz - 1 - BZ >= 0 ? (G.nz - 1 - BZ) / BZ : 0;
  return ts;
}
inline bool pipelined_tiles(const Geom& G) {
  const bool mirror_x = (G.bc[0] == BC_FREESLIP || G.bc[0] == BC_INFLOW_WALL) &&
                        (G.bc[1] == BC_FREESLIP || G.bc[1] == BC_INFLOW_WALL);
  return mirror_x && !(G.nx & 1) && default_tile_split(G).interior() > 0;
}

// dmap, tma: with tma != 0 (two-pass kernels with an FP32 tile), the tensor map of the pass-1
// field (rho, phi) as 8-byte cells over (x, y, z + 1), planes z = -1 .. nz, box 36 x TY x TZ; the
// block's tile then arrives by one TMA copy while the population loads are in flight.  bmode != 0:
// a one-dimensional grid over the boundary tiles of bt (the pipelined kernel takes the others).
template <class Store, int MINB, bool FUSED, class B = BlkDefault>
__global__ void __launch_bounds__(B::NT, MINB)
    k_collide_stream(Store st, const __grid_constant__ Geom G,
                     const __grid_constant__ KConst<typename DensOf<Store>::real> K, int odd,
                     const typename DensOf<Store>::type* __restrict__ dens, long long* __restrict__ counter,
                     const FusedIO io, const __grid_constant__ CUtensorMap dmap, int tma, const TileSplit bt,
                     int bmode) {
  using R = typename DensOf<Store>::real;  // compute type: FP64 for FP64 storage, FP32 otherwise
  using DT = typename DensOf<Store>::type;
  __shared__ __align__(128) DT tile[B::TILET];
  __shared__ float2 prow[FUSED ? B::NW * 9 * B::TX : 1];
  __shared__ int pfast[B::NW];
  __shared__ uint64_t tbar;

  int x0 = blockIdx.x * B::BX, y0 = blockIdx.y * B::BY, z0 = blockIdx.z * B::BZ;
  if (bmode) {
    // the block's boundary tile, computed once (block 0: the tile at the origin)
    __shared__ int3 btile;
    if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
      int a, b, c;
      bt.boundary_tile(blockIdx.x, B::BY, B::BZ, a, b, c);
      btile = make_int3(a, b, c);
    }
    __syncthreads();
    x0 = btile.x;
    y0 = btile.y;
    z0 = btile.z;
  }
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
  const bool active = x < G.nx && y < G.ny && z < G.nz;
  const int tid = threadIdx.x + B::BX * (threadIdx.y + B::BY * threadIdx.z);
  const long long step = counter[odd];
  if (tid == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) counter[odd ^ 1] = step + 1;

  // block-uniform: the tile comes by TMA (no periodic face crossed)
  bool via_tma = false;
  if constexpr (!FUSED && std::is_same<DT, float2>::value) {
    via_tma = tma != 0 && !tile_wraps<B>(G, x0, y0, z0);
    if (via_tma) {
      if (tid == 0) {
        mbar_init(&tbar, 1);
        mbar_fence_init();
        mbar_arrive_expect_tx(&tbar, (uint32_t)(B::TILET * sizeof(DT)));
        tma_load_3d(tile, &dmap, &tbar, x0 - 2, y0 - 1, z0);  // tensor plane z0 is z = z0 - 1
      }
      __syncthreads();  // the initialised barrier is visible to every thread before it waits
    }
  }

  R rho_r = R(0), ft[27];
  // a warp is one x-row of the block: the fast-row test is warp-uniform (the fused pass sums
  // across the 32 lanes of a fast row, so there the row must also be complete in x)
  const bool fast = fast_row(G, y, z) && (!FUSED || x0 + B::BX <= G.nx);
  if (FUSED && threadIdx.x == 0) pfast[tid >> 5] = active && fast;
  if (active) {
    if (fast) {
      AoRow ar;  // rebuilt for the stores: cheaper than keeping it live through the collision
      ar.init<Store::PLANES>(G, x, y, z);
      load_node_fast(st, K, G, ar, odd, rho_r, ft);
    } else {
      NodeMap nm;
      nm.init(G, x, y, z);
      load_node(st, K, nm, odd, rho_r, ft);
    }
  }

  if (via_tma) {
    // every thread waits for the copy (the barrier's phase completes with the copy's bytes), then
    // the out-of-box cells get their mirror ghosts; a wait that runs out flags LBM_ETIMEOUT (the
    // step's result is not used) and the copy's issuer waits once more before the block leaves
    if (!mbar_wait(&tbar, 0)) {
      atomicOr(io.flag, kFlagTimeout);
      if (tid == 0) mbar_wait(&tbar, 0);
    }
    TileRange tr;
    tr.init<B>(G, x0, y0, z0);
    if (tr.clamps<B>()) {
      tile_clamp_fix<B>(tile, tr, tid);
      __syncthreads();
    }
  } else {
    // halo tile of (rho, phi) by loads: warp w fills rows w, w+8, w+16, ... of the TY*TZ rows of
    // columns 1..34 (x0-1 .. x0+32); lanes cover x0-1 .. x0+30 and lanes 0..1 also x0+31, x0+32.
    const int warp = tid >> 5, lane = threadIdx.x;
    const int xa = wrap_or_clamp(x0 + lane - 1, G.nx, G.bc[0], G.bc[1]);
    const int xb = wrap_or_clamp(x0 + lane + 31, G.nx, G.bc[0], G.bc[1]);
    const int cxa = xa < G.nx ? xa : G.nx - 1, cxb = xb < G.nx ? xb : G.nx - 1;
    const float rho_r0f = (float)K.rho_r0_d;
#pragma unroll
    for (int k = 0; k < (B::TY * B::TZ + B::NT / 32 - 1) / (B::NT / 32); ++k) {
      const int row = warp + k * (B::NT / 32);
      if (row < B::TY * B::TZ) {
        const int ty = row % B::TY, tz = row / B::TY;
        const int gy = wrap_or_clamp(y0 + ty - 1, G.ny, G.bc[2], G.bc[3]);
        const int gz = wrap_or_clamp(z0 + tz - 1, G.nz, G.bc[4], G.bc[5]);
        // out-of-box tail rows of a ragged block read a clamped in-box row
        const int cy = gy < G.ny ? gy : G.ny - 1, cz = gz <= tile_zmax(G) ? gz : tile_zmax(G);
        const int64_t rbase = (int64_t)G.nx * ((int64_t)cy + (int64_t)G.ny * cz);
        if constexpr (FUSED) {
          tile[row * B::TXT + 1 + lane] = fused_cell(io, rbase + cxa);
          if (lane < B::TX - 32) tile[row * B::TXT + 33 + lane] = fused_cell(io, rbase + cxb);
        } else {
          tile[row * B::TXT + 1 + lane] = dens[rbase + cxa];
          if (lane < B::TX - 32) tile[row * B::TXT + 33 + lane] = dens[rbase + cxb];
        }
      }
    }
    if constexpr (FUSED) {
      if (G.inflow && z0 <= 1) {
        // the Dirichlet inlet nodes carry rho_r0 and phi = 1, as in pass 1: in the tile planes that
        // read the z = 0 plane (for z0 = 0: plane 0, the mirror ghost z = -1, and plane 1; for
        // z0 = 1, which 32 x BY x 1 blocks reach: plane 0).  Block-uniform branch.
        __syncthreads();
        for (int c = tid; c < B::TX * B::TY; c += B::NT) {
          int gx = wrap_or_clamp(x0 + c % B::TX - 1, G.nx, G.bc[0], G.bc[1]);
          int gy = wrap_or_clamp(y0 + c / B::TX - 1, G.ny, G.bc[2], G.bc[3]);
          gx = gx < G.nx ? gx : G.nx - 1;
          gy = gy < G.ny ? gy : G.ny - 1;
          if (is_inlet(G, gx, gy, 0)) {
            const int ct = c % B::TX + 1 + B::TXT * (c / B::TX);  // the cell's index in the tile
            tile[ct] = make_float2(rho_r0f, 1.0f);  // plane 0: z = -1 (z0 = 0) or z = 0 (z0 = 1)
            if (z0 == 0) tile[ct + B::TXT * B::TY] = make_float2(rho_r0f, 1.0f);
          }
        }
      }
    }
    __syncthreads();
  }
  if (!FUSED && !active) return;

  if (active) {
    R gphi[3], grho[3];
    tile_gradients<R, DT, B::TXT, B::TY>(tile, threadIdx.x + 2, threadIdx.y + 1, threadIdx.z + 1, gphi, grho);

    R f[27];
    Recol<R> rc;
    if (is_inlet(G, x, y, z)) {
      inlet_state(K, dnode(G, x, y, z), (int64_t)step, f);
      rc.frac = R(1);
      rc.n0 = rc.n1 = rc.n2 = R(0);
      rc.rc[0] = rc.rc[1] = rc.rc[2] = rc.rc[3] = R(0);
      rc.rho = R(1);
      rc.has_n = false;
    } else {
      rc = collide(K, rho_r, ft, gphi, grho, f);
    }
    if constexpr (FUSED) {
      // the watchdog of pass 1, on the density this step starts from
      if (!(rc.rho > R(0)) || !(rc.rho < R(1e30))) atomicOr(io.flag, 1);
    }
    // warp-uniform: does any node of the warp carry an interface normal?
    const bool recol = __any_sync(__activemask(), any_(rc.has_n));
    NodeMap nm;
    AoRow ar;
    if (fast) {
      ar.init<Store::PLANES>(G, x, y, z);
      // the parity as a template argument: no per-direction branch on it in the stores (the
      // fused density pass keeps it a runtime value: the extra code raised its spills)
      if constexpr (FUSED) {
        if (recol) EmitLoop<0, Store, R, true, true, FUSED, -1, B::BY, B::TX>::run(st, K, G, nm, ar, odd != 0, f, rc, prow, io, x, y, z);
        else EmitLoop<0, Store, R, true, false, FUSED, -1, B::BY, B::TX>::run(st, K, G, nm, ar, odd != 0, f, rc, prow, io, x, y, z);
      } else if (recol) {
        if (odd) EmitLoop<0, Store, R, true, true, FUSED, 1, B::BY, B::TX>::run(st, K, G, nm, ar, true, f, rc, prow, io, x, y, z);
        else EmitLoop<0, Store, R, true, true, FUSED, 0, B::BY, B::TX>::run(st, K, G, nm, ar, false, f, rc, prow, io, x, y, z);
      } else {
        if (odd) EmitLoop<0, Store, R, true, false, FUSED, 1, B::BY, B::TX>::run(st, K, G, nm, ar, true, f, rc, prow, io, x, y, z);
        else EmitLoop<0, Store, R, true, false, FUSED, 0, B::BY, B::TX>::run(st, K, G, nm, ar, false, f, rc, prow, io, x, y, z);
      }
    } else {
      if (odd) nm.init(G, x, y, z);
      else nm.base = snode(G, x, y, z);  // the even step only uses the base
      if (recol) EmitLoop<0, Store, R, false, true, FUSED, -1, B::BY, B::TX>::run(st, K, G, nm, ar, odd != 0, f, rc, prow, io, x, y, z);
      else EmitLoop<0, Store, R, false, false, FUSED, -1, B::BY, B::TX>::run(st, K, G, nm, ar, odd != 0, f, rc, prow, io, x, y, z);
    }
  }

  if constexpr (FUSED) {
    // merge the warps' rows into the global accumulators: tile row (ty, tz) (target y = y0-1+ty,
    // z = z0-1+tz) sums, in a fixed order, row K = (ty-wy) + 3(tz-wz) of every fast warp (wy, wz)
    // within one row of it; warp w takes tile rows w, w+8, w+16, lanes the columns
    __syncthreads();
    const int warp = tid >> 5, lane = threadIdx.x;
    int gxa = x0 - 1 + lane, gxb = x0 + 31 + lane;  // lanes 0..1 also take columns 32, 33
    if (gxa < 0) gxa = G.bc[0] == BC_PERIODIC ? G.nx - 1 : 0;
    if (gxb >= G.nx) gxb = G.bc[1] == BC_PERIODIC ? gxb - G.nx : G.nx - 1;
    const bool ina = gxa < G.nx, inb = lane < B::TX - 32 && gxb >= 0 && gxb < G.nx;
#pragma unroll
    for (int k = 0; k < (B::TY * B::TZ + B::NW - 1) / B::NW; ++k) {
      const int row = warp + k * B::NW;
      if (row < B::TY * B::TZ) {
        const int ty = row % B::TY, tz = row / B::TY;
        const int gy = y0 - 1 + ty, gz = z0 - 1 + tz;
        if (gy >= 0 && gy < G.ny && gz >= 0 && gz < G.nz) {
          float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
#pragma unroll
          for (int wz = 0; wz < B::BZ; ++wz) {
#pragma unroll
            for (int wy = 0; wy < B::BY; ++wy) {
              const int ky = ty - wy, kz = tz - wz;
              if (ky >= 0 && ky <= 2 && kz >= 0 && kz <= 2 && pfast[wy + B::BY * wz]) {
                const float2* src = prow + ((wy + B::BY * wz) * 9 + ky + 3 * kz) * B::TX;
                const float2 u = src[lane];
                a.x += u.x;
                a.y += u.y;
                if (lane < B::TX - 32) {
                  const float2 v = src[32 + lane];
                  b.x += v.x;
                  b.y += v.y;
                }
              }
            }
          }
          const int64_t rb = (int64_t)G.nx * ((int64_t)gy + (int64_t)G.ny * gz);
          const unsigned long long av = pack_fix(a.x, a.y), bv = pack_fix(b.x, b.y);
          if (ina && av) atomicAdd(io.nxt + rb + gxa, av);
          if (inb && bv) atomicAdd(io.nxt + rb + gxb, bv);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// pass 2, software-pipelined (packed storage).  A persistent block walks over
// the tiles of the box; while it computes one tile, the next tile's population
// words (the same slots the one-node kernel loads) and its (rho, phi) halo are
// already on their way into shared memory through asynchronous copies
// (cp.async), so the collision does not wait on memory latency.  Two stages
// of 27 x 256 words + the halo tile: 68 KB per block, 3 blocks per SM.
constexpr int PF_POP = 27 * NTHREADS;
constexpr int PF_STAGE_BYTES = PF_POP * 4 + TILE * 8;
constexpr int PF_SMEM = 2 * PF_STAGE_BYTES;

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// word index of direction t's post-streaming value of a node on a fast row (step parity odd)
template <int T>
__device__ __forceinline__ int64_t fast_src(const Geom& G, const AoRow& ar, int odd) {
  if (!odd) return ar.e[1] + T * 32;
  return ar.slot0<26 - T, 27>(G) + (26 - T) * 32;
}
template <int T>
struct PfIssueFast {
  __device__ __forceinline__ static void run(const uint32_t* A, const Geom& G, const AoRow& ar, int odd,
                                             uint32_t* pop_s, int tid) {
    cp_async4(pop_s + T * NTHREADS + tid, A + fast_src<T>(G, ar, odd));
    PfIssueFast<T + 1>::run(A, G, ar, odd, pop_s, tid);
  }
};
template <>
struct PfIssueFast<27> {
  __device__ __forceinline__ static void run(const uint32_t*, const Geom&, const AoRow&, int, uint32_t*, int) {}
};

// start the copies of tile (x0, y0, z0) into one stage
__device__ __forceinline__ void pf_issue(const uint32_t* A, const Geom& G, const float2* __restrict__ dens, int odd,
                                         int x0, int y0, int z0, uint32_t* pop_s, float2* tile_s) {
  const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
  if (x < G.nx && y < G.ny && z < G.nz) {
    if (fast_row(G, y, z)) {
      AoRow ar;
      ar.init<27>(G, x, y, z);
      PfIssueFast<0>::run(A, G, ar, odd, pop_s, tid);
    } else {
      NodeMap nm;
      nm.init(G, x, y, z);
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        int64_t node;
        int dir;
        slot_of(nm, odd, t, node, dir);
        cp_async4(pop_s + t * NTHREADS + tid, A + elem_index(node, 27, dir));
      }
    }
  }
  const int warp = tid >> 5, lane = threadIdx.x;
  const int xa = wrap_or_clamp(x0 + lane - 1, G.nx, G.bc[0], G.bc[1]);
  const int xb = wrap_or_clamp(x0 + lane + 31, G.nx, G.bc[0], G.bc[1]);
  const int cxa = xa < G.nx ? xa : G.nx - 1, cxb = xb < G.nx ? xb : G.nx - 1;
#pragma unroll
  for (int k = 0; k < (TY * TZ + NWARPS - 1) / NWARPS; ++k) {
    const int row = warp + k * NWARPS;
    if (row < TY * TZ) {
      const int gy = wrap_or_clamp(y0 + row % TY - 1, G.ny, G.bc[2], G.bc[3]);
      const int gz = wrap_or_clamp(z0 + row / TY - 1, G.nz, G.bc[4], G.bc[5]);
      const int64_t rbase = (int64_t)G.nx * ((int64_t)(gy < G.ny ? gy : G.ny - 1) +
                                              (int64_t)G.ny * (gz <= tile_zmax(G) ? gz : tile_zmax(G)));
      cp_async8(tile_s + row * TX + lane, dens + rbase + cxa);
      if (lane < TX - 32) cp_async8(tile_s + row * TX + 32 + lane, dens + rbase + cxb);
    }
  }
}

template <class Store, int MINB>
__global__ void __launch_bounds__(NTHREADS, MINB)
    k_collide_stream_pf(Store st, const __grid_constant__ Geom G, const __grid_constant__ KConst<float> K, int odd,
                        const float2* __restrict__ dens, long long* __restrict__ counter, int ntx, int nty,
                        int ntiles) {
  static_assert(Store::PLANES == 27, "packed storage only");
  extern __shared__ __align__(16) unsigned char pf_smem[];
  // stage k: words at pf_smem + k * PF_STAGE_BYTES, halo tile after them
#define PF_POP_S(k) reinterpret_cast<uint32_t*>(pf_smem + (k) * PF_STAGE_BYTES)
#define PF_TILE_S(k) reinterpret_cast<float2*>(pf_smem + (k) * PF_STAGE_BYTES + PF_POP * 4)
  const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
  const long long step = counter[odd];  // step index protocol of k_collide_stream
  if (tid == 0 && blockIdx.x == 0) counter[odd ^ 1] = step + 1;

  int tile = blockIdx.x;
  if (tile < ntiles)
    pf_issue(st.A, G, dens, odd, (tile % ntx) * BX, ((tile / ntx) % nty) * BY, (tile / (ntx * nty)) * BZ,
             PF_POP_S(0), PF_TILE_S(0));
  cp_async_commit();
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const int nxt = tile + gridDim.x;
    if (nxt < ntiles)
      pf_issue(st.A, G, dens, odd, (nxt % ntx) * BX, ((nxt / ntx) % nty) * BY, (nxt / (ntx * nty)) * BZ,
               PF_POP_S((it + 1) & 1), PF_TILE_S((it + 1) & 1));
    cp_async_commit();
    cp_async_wait_prev();  // this tile's copies (all but the group just issued) have landed
    __syncthreads();
    const uint32_t* ps = PF_POP_S(it & 1);
    const float2* ts = PF_TILE_S(it & 1);
    const int x0 = (tile % ntx) * BX, y0 = ((tile / ntx) % nty) * BY, z0 = (tile / (ntx * nty)) * BZ;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    if (x < G.nx && y < G.ny && z < G.nz) {
      float rho_r = 0.0f, ft[27];
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        float fr;
        Store::decode(ps[t * NTHREADS + tid], K.refB[speed2_of(t)], speed2_of(t) == 0 ? K.dref[0] : 0.0f, fr, ft[t]);
        rho_r += fr;
      }
      float gphi[3], grho[3];
      tile_gradients<float>(ts, threadIdx.x + 1, threadIdx.y + 1, threadIdx.z + 1, gphi, grho);
      float f[27];
      Recol<float> rc;
      if (is_inlet(G, x, y, z)) {
        inlet_state(K, dnode(G, x, y, z), (int64_t)step, f);
        rc.frac = 1.0f;
        rc.n0 = rc.n1 = rc.n2 = 0.0f;
        rc.rc[0] = rc.rc[1] = rc.rc[2] = rc.rc[3] = 0.0f;
        rc.rho = 1.0f;
        rc.has_n = false;
      } else {
        rc = collide(K, rho_r, ft, gphi, grho, f);
      }
      const bool recol = __any_sync(__activemask(), rc.has_n);
      const bool fast = fast_row(G, y, z);
      NodeMap nm;
      AoRow ar;
      FusedIO io{};
      if (fast) {
        ar.init<27>(G, x, y, z);
        if (recol) EmitLoop<0, Store, float, true, true, false>::run(st, K, G, nm, ar, odd != 0, f, rc, nullptr, io, x, y, z);
        else EmitLoop<0, Store, float, true, false, false>::run(st, K, G, nm, ar, odd != 0, f, rc, nullptr, io, x, y, z);
      } else {
        if (odd) nm.init(G, x, y, z);
        else nm.base = snode(G, x, y, z);
        if (recol) EmitLoop<0, Store, float, false, true, false>::run(st, K, G, nm, ar, odd != 0, f, rc, nullptr, io, x, y, z);
        else EmitLoop<0, Store, float, false, false, false>::run(st, K, G, nm, ar, odd != 0, f, rc, nullptr, io, x, y, z);
      }
    }
    __syncthreads();  // the stage is refilled in the next iteration
  }
#undef PF_POP_S
#undef PF_TILE_S
}

// ---------------------------------------------------------------------------
// pass 2, two nodes per thread (FP32 arithmetic on both lanes at once).
// Block: 16 x 4 x 2 threads over 32 x 4 x 2 nodes; thread tx owns the node
// pair (x0 + 2tx, x0 + 2tx + 1).  Needs nx even, so a pair is never split by
// the box and the even node's storage index is even (8-byte aligned pairs).
constexpr int PX = 16, PY = BY, PZ = BZ;
constexpr int PTHREADS = PX * PY * PZ;

template <int T, class Store>
__device__ __forceinline__ void emit2(const Store& st, const KConst<F2>& K, int64_t base, const NodeMap& m0,
                                      const NodeMap& m1, bool odd, const F2 f[27], const Recol<F2>& rc) {
  constexpr int cls = speed2_of(T);
  const float rB = K.refB[cls].v.x, dR = cls == 0 ? K.dref[0].v.x : 0.0f;
  const F2 fstar = f[T];
  F2 outr, q;
  if (T == REST) {
    outr = rc.frac * fstar;
    q = rc.frac;
  } else {
    const F2 cn = cdot<T>(rc.n0, rc.n1, rc.n2);
    outr = fma_(rc.frac, fstar, rc.rc[cls] * cn);
    q = select_(rc.has_n, sat_(outr * rcp_(fstar)), rc.frac);
  }
  const F2 outb = fstar - outr;
  if (!odd) {
    st.store_p(base, opp_of(T), rB, dR, outr, outb, fstar, q);
  } else {
    int64_t n0, n1;
    int d0, d1;
    m0.push<T>(n0, d0);
    m1.push<T>(n1, d1);
    st.store_s(n0, d0, rB, dR, outr.v.x, outb.v.x, fstar.v.x, q.v.x);
    st.store_s(n1, d1, rB, dR, outr.v.y, outb.v.y, fstar.v.y, q.v.y);
  }
}

template <int T, class Store>
struct EmitLoop2 {
  __device__ __forceinline__ static void run(const Store& st, const KConst<F2>& K, int64_t base, const NodeMap& m0,
                                             const NodeMap& m1, bool odd, const F2* f, const Recol<F2>& rc) {
    emit2<T>(st, K, base, m0, m1, odd, f, rc);
    EmitLoop2<T + 1, Store>::run(st, K, base, m0, m1, odd, f, rc);
  }
};
template <class Store>
struct EmitLoop2<27, Store> {
  __device__ __forceinline__ static void run(const Store&, const KConst<F2>&, int64_t, const NodeMap&,
                                             const NodeMap&, bool, const F2*, const Recol<F2>&) {}
};

template <class Store, int MINB>
__global__ void __launch_bounds__(PTHREADS, MINB)
    k_collide_stream2(Store st, const __grid_constant__ Geom G, const __grid_constant__ KConst<F2> K, int odd,
                      const float2* __restrict__ dens, long long* __restrict__ counter) {
  __shared__ float2 tile[TILE];
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * PY, z0 = blockIdx.z * PZ;
  const long long step = counter[odd];  // step index protocol of k_collide_stream
  if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0 && blockIdx.x == 0 && blockIdx.y == 0 &&
      blockIdx.z == 0)
    counter[odd ^ 1] = step + 1;
  const int xa = x0 + 2 * threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
  const bool active = xa < G.nx && y < G.ny && z < G.nz;  // nx even: xa + 1 < nx as well

  const int64_t base = snode(G, xa, y, z);
  NodeMap m0, m1;
  F2 rho_r = F2(0.0f), ft[27];
  if (active) {
    if (!odd) {
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        F2 fr;
        st.load_p(base, t, K.refB[speed2_of(t)].v.x, speed2_of(t) == 0 ? K.dref[0].v.x : 0.0f, fr, ft[t]);
        rho_r = rho_r + fr;
      }
    } else {
      m0.init(G, xa, y, z);
      m1.init(G, xa + 1, y, z);
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        int64_t n0, n1;
        int d0, d1;
        slot_of(m0, 1, t, n0, d0);
        slot_of(m1, 1, t, n1, d1);
        const float rB = K.refB[speed2_of(t)].v.x, dR = speed2_of(t) == 0 ? K.dref[0].v.x : 0.0f;
        F2 fr;
        st.load_s(n0, d0, rB, dR, fr.v.x, ft[t].v.x);
        st.load_s(n1, d1, rB, dR, fr.v.y, ft[t].v.y);
        rho_r = rho_r + fr;
      }
    }
  }

  // halo tile of (rho, phi): warp w fills rows w, w+4, ... of the TY*TZ rows
  {
    const int tid = threadIdx.x + PX * (threadIdx.y + PY * threadIdx.z);
    const int warp = tid >> 5, lane = tid & 31;
    const int xl = wrap_or_clamp(x0 + lane - 1, G.nx, G.bc[0], G.bc[1]);
    const int xr = wrap_or_clamp(x0 + lane + 31, G.nx, G.bc[0], G.bc[1]);
    const int cxl = xl < G.nx ? xl : G.nx - 1, cxr = xr < G.nx ? xr : G.nx - 1;
#pragma unroll
    for (int k = 0; k < (TY * TZ + PTHREADS / 32 - 1) / (PTHREADS / 32); ++k) {
      const int row = warp + k * (PTHREADS / 32);
      if (row < TY * TZ) {
        const int ty = row % TY, tz = row / TY;
        const int gy = wrap_or_clamp(y0 + ty - 1, G.ny, G.bc[2], G.bc[3]);
        const int gz = wrap_or_clamp(z0 + tz - 1, G.nz, G.bc[4], G.bc[5]);
        const int64_t rbase = (int64_t)G.nx * ((int64_t)(gy < G.ny ? gy : G.ny - 1) +
                                                (int64_t)G.ny * (gz <= tile_zmax(G) ? gz : tile_zmax(G)));
        tile[row * TX + lane] = dens[rbase + cxl];
        if (lane < TX - 32) tile[row * TX + 32 + lane] = dens[rbase + cxr];
      }
    }
  }
  __syncthreads();
  if (!active) return;

  F2 gphi[3] = {F2(0.0f), F2(0.0f), F2(0.0f)}, grho[3] = {F2(0.0f), F2(0.0f), F2(0.0f)};
  const int lx = 2 * threadIdx.x + 1, ly = threadIdx.y + 1, lz = threadIdx.z + 1;
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    if (t == REST) continue;
    const int o = (lx + cx_of(t)) + TX * ((ly + cy_of(t)) + TY * (lz + cz_of(t)));
    const float2 v0 = tile[o], v1 = tile[o + 1];
    const F2 w3 = F2(float(3.0 * weight_of(t)));
    const F2 a = w3 * F2(v0.y, v1.y), b = w3 * F2(v0.x, v1.x);
    if (cx_of(t) != 0) { gphi[0] = fma_(F2(float(cx_of(t))), a, gphi[0]); grho[0] = fma_(F2(float(cx_of(t))), b, grho[0]); }
    if (cy_of(t) != 0) { gphi[1] = fma_(F2(float(cy_of(t))), a, gphi[1]); grho[1] = fma_(F2(float(cy_of(t))), b, grho[1]); }
    if (cz_of(t) != 0) { gphi[2] = fma_(F2(float(cz_of(t))), a, gphi[2]); grho[2] = fma_(F2(float(cz_of(t))), b, grho[2]); }
  }

  F2 f[27];
  Recol<F2> rc = collide(K, rho_r, ft, gphi, grho, f);
  if (z == 0 && G.inflow) {
    // Dirichlet inlet nodes (Sec. IV.A) replace the collision result lane by lane
#pragma unroll
    for (int lane = 0; lane < 2; ++lane) {
      if (is_inlet(G, xa + lane, y, z)) {
        float fin[27];
        KConst<float> Ks;
        Ks.u_j0 = K.u_j0;
        Ks.noise_frac = K.noise_frac;
        Ks.seed = K.seed;
        Ks.rho_r0_d = K.rho_r0_d;
        Ks.alpha_r_d = K.alpha_r_d;
        inlet_state(Ks, dnode(G, xa + lane, y, z), (int64_t)step, fin);
#pragma unroll
        for (int t = 0; t < 27; ++t) {
          if (lane == 0) f[t].v.x = fin[t]; else f[t].v.y = fin[t];
        }
        if (lane == 0) {
          rc.frac.v.x = 1.0f; rc.n0.v.x = rc.n1.v.x = rc.n2.v.x = 0.0f; rc.has_n.x = false;
          rc.rc[1].v.x = rc.rc[2].v.x = rc.rc[3].v.x = 0.0f;
        } else {
          rc.frac.v.y = 1.0f; rc.n0.v.y = rc.n1.v.y = rc.n2.v.y = 0.0f; rc.has_n.y = false;
          rc.rc[1].v.y = rc.rc[2].v.y = rc.rc[3].v.y = 0.0f;
        }
      }
    }
  }
  EmitLoop2<0, Store>::run(st, K, base, m0, m1, odd != 0, f, rc);
}


// sum over the 32 lanes of a warp, the same value in every lane (butterfly: lanes i and i^o
// hold the same partial sum at every stage, as addition commutes exactly)
template <typename R>
__device__ __forceinline__ R warp_allsum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// convective outflow on the z = nz-1 plane (Sec. IV.A), after the step that
// produced time t+1; `layout` is the layout of time t+1.  One warp per column
// (x, y), lane t < 27 for direction t (the plane holds only nx ny nodes: a
// thread per node would leave most of the SMs idle and run each column's 27
// directions one after another); the slot map uses selects, so the lanes do not
// diverge.  The lanes reduce rho and the z momentum of the node below with
// shuffles, then each sets f(N, t+1) = (f(N, t) + lambda f(N-1, t+1)) /
// (1 + lambda) for its direction and both colours, lambda = max(0, u_z(N-1, t+1));
// `top` holds f(N, t) per column (32 red then 32 blue slots), and is updated.
template <class Store>
__global__ void __launch_bounds__(256) k_outflow(Store st, Geom G,
                                                 const __grid_constant__ KConst<typename DensOf<Store>::real> K,
                                                 int layout, typename DensOf<Store>::real* __restrict__ top,
                                                 unsigned long long* __restrict__ fix) {
  using R = typename DensOf<Store>::real;
  const int64_t Pn = (int64_t)G.nx * G.ny;
  const int64_t pp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;  // warp-uniform
  if (pp >= Pn) return;
  const int lane = threadIdx.x & 31;
  const bool act = lane < 27;
  const int t = act ? lane : 0;
  const int x = (int)(pp % G.nx), y = (int)(pp / G.nx);
  NodeMap below, here;
  below.init(G, x, y, G.nz - 2);
  here.init(G, x, y, G.nz - 1);
  R fr = R(0), fb = R(0);
  if (act) {
    int64_t node;
    int dir;
    slot_of_rt(below, layout, t, node, dir);
    st.load_rb(node, dir, speed2_of(t), K, fr, fb);
  }
  const R v = fr + fb;
  const R rho = warp_allsum(v);
  const R mz = warp_allsum(cz_of(t) > 0 && act ? v : cz_of(t) < 0 && act ? -v : R(0));
  R F[3];
  body_force(K, rho, F);
  const R uz = (mz + R(0.5) * F[2]) / rho;
  const R lam = uz > R(0) ? uz : R(0);
  const R inv = R(1) / (R(1) + lam);
  R nr = R(0), nb = R(0);
  if (act) {
    R* tr = top + pp * 64 + t;  // per column: 32 red then 32 blue slots, one line per warp
    R* tb = tr + 32;
    nr = (*tr + lam * fr) * inv;
    nb = (*tb + lam * fb) * inv;
    *tr = nr;
    *tb = nb;
    int64_t node;
    int dir;
    slot_of_rt(here, layout, t, node, dir);
    store_pair(st, K, node, dir, nr, nb);
  }
  // fused density pass: the plane's new populations replace what the collide-stream kernel accumulated
  if (fix) {
    const R sr = warp_allsum(nr), sa = warp_allsum(nr + nb);
    if (lane == 0) fix[dnode(G, x, y, G.nz - 1)] = pack_fix((float)sa, (float)sr);
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
#pragma unroll
  for (int t = 0; t < 27; ++t) {  // the lattice constants fold at compile time
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
  st.load_rb(node, dir, speed2_of(t), K, fr, fb);
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
    st.load_rb(node, dir, speed2_of(t), K, fr, fb);
    top[pp * 64 + t] = fr;  // per column: 32 red then 32 blue slots (27 used)
    top[pp * 64 + 32 + t] = fb;
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
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    int64_t node;
    int dir;
    slot_of(nm, layout, t, node, dir);
    st.load_rb(node, dir, speed2_of(t), K, fr[t], fb[t]);
  }
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
