// Compact 16-bit storage: the total population per direction plus one colour record per node
// (templates; instantiated in lbm_kernels_c16.cu).
//
// The recolouring of Sec. II hands every node's post-collision populations to the two colours
// by one rule for all directions:
//   f^r_i = (rho_r/rho) f*_i + beta (rho_r rho_b/rho^2) cos(theta_i) rho varphi_i(alpha_bar)
//         = frac f*_i + (w_i/|c_i|) (c_i . m),     m = beta rho_r rho_b/rho (27/19)(1 - alpha_bar) n,
// (varphi_i(alpha) = (27/19)(1 - alpha) w_i for the moving directions, cos(theta_rest) = 0), so
// the colour split of everything a node emits is fixed by four numbers, the record
// (frac, m_x, m_y, m_z).  The storage keeps, per node, the total post-collision population of
// every direction and the node's record; the red population in any slot is rebuilt from the
// slot's total and the record of the node that emitted it (the owner of S(x, opp(i)), the
// direction it left along opp(stored direction), see lbm_kernels.cuh).  Only the red density
// per node is ever needed (the collision acts on the total), so pass 1 rebuilds the colour
// split once per population and pass 2 does not rebuild it at all: it takes rho_r from the
// (rho, phi) field of pass 1.
//
// Layout: blocks of 32 storage nodes, 28 planes of 32 unsigned 16-bit words each.  Plane t
// (tensor order, t != 13) holds direction t's total as a half / bfloat16 deviation from the
// direction's rest value rho_b0 w_t, which the density-ratio relation of Sec. II makes the
// same in both pure phases for every moving direction; planes 13 and 27 hold the high and low
// halves of the rest direction's total in FP32.  56 bytes per node, then one float4 record per
// storage node (16 bytes).
//
// The state set by lbm_init_fields or lbm_set_populations (per-colour equilibria or arbitrary
// per-colour populations) has no record form; the host then writes (rho, phi) directly and the
// first step skips pass 1.  The top plane of an outflow face is replaced per colour by the
// convective outflow update, which has no record form either: its populations live, per
// colour, in the outflow history buffer (Geom::ctop), which every kernel reads for that plane.
#pragma once
#include "lbm_kernels.cuh"

namespace lbmk {

constexpr int CPLANES = 28;            // 16-bit planes per block
constexpr int REST_HI = 13, REST_LO = 27;

template <bool BF16>
struct CompactStore {
  static constexpr int PLANES = CPLANES;  // AoRow / slot addressing in 16-bit units
  uint16_t* A;
  float4* rec;
  int64_t Ns;

  __device__ __forceinline__ static float dev_to_float(uint16_t bits) {
    if (BF16) return __uint_as_float((uint32_t)bits << 16);
    return __half2float(__ushort_as_half(bits));
  }
  __device__ __forceinline__ static uint16_t float_to_dev(float v) {
    if (BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    return __half_as_ushort(__float2half_rn(v));
  }
  // total population of stored direction `dir` (speed class cls) of the slot with plane-0 index e0
  __device__ __forceinline__ float load_at(int64_t e0, int dir, int cls, const KConst<float>& K) const {
    if (dir == REST) {
      const uint32_t hi = __ldcs(A + e0 + REST_HI * 32), lo = __ldcs(A + e0 + REST_LO * 32);
      return __uint_as_float((hi << 16) | lo);
    }
    return K.refB[cls] + dev_to_float(__ldcs(A + e0 + dir * 32));
  }
  __device__ __forceinline__ void store_at(int64_t e0, int dir, int cls, const KConst<float>& K, float f) const {
    if (dir == REST) {
      const uint32_t b = __float_as_uint(f);
      __stcs(A + e0 + REST_HI * 32, (uint16_t)(b >> 16));
      __stcs(A + e0 + REST_LO * 32, (uint16_t)(b & 0xFFFFu));
      return;
    }
    __stcs(A + e0 + dir * 32, float_to_dev(f - K.refB[cls]));
  }
  __device__ __forceinline__ float load(int64_t node, int dir, int cls, const KConst<float>& K) const {
    return load_at(elem_index(node, CPLANES, 0), dir, cls, K);
  }
  __device__ __forceinline__ void store(int64_t node, int dir, int cls, const KConst<float>& K, float f) const {
    store_at(elem_index(node, CPLANES, 0), dir, cls, K, f);
  }
};

// w_s / |c| of speed class s: the weight of c_i . m in the colour split of a moving direction
__device__ __forceinline__ float split_coef(int cls) {
  return cls == 1 ? (float)(2.0 / 27.0) : cls == 2 ? (float)(1.0 / 54.0 * 0.70710678118654752440)
                                                   : (float)(1.0 / 216.0 * 0.57735026918962576451);
}

// c_t . (a0, a1, a2) by signed additions (t known at compile time after unrolling: the zero
// components vanish; -0 is the exact identity of addition)
__device__ __forceinline__ float cdot_c(int t, float a0, float a1, float a2) {
  float s = -0.0f;
  if (cx_of(t) > 0) s += a0;
  if (cx_of(t) < 0) s -= a0;
  if (cy_of(t) > 0) s += a1;
  if (cy_of(t) < 0) s -= a1;
  if (cz_of(t) > 0) s += a2;
  if (cz_of(t) < 0) s -= a2;
  return s;
}

// red part of a slot: total f, record r of the emitting node, direction j it left along
__device__ __forceinline__ float red_of(float f, const float4& r, int j) {
  if (j == REST) return r.x * f;
  const float cm = (float)cx_of(j) * r.y + (float)cy_of(j) * r.z + (float)cz_of(j) * r.w;
  return fmaf(split_coef(speed2_of(j)), cm, r.x * f);
}

__device__ __forceinline__ bool on_top(const Geom& G, int z) { return G.ctop != nullptr && z == G.nz - 1; }

// loads of the 27 totals of a node on a fast row: direction t in layout 0 from the node's own
// slot t, in layout 1 from the slot S(x, opp(t))
template <int LAYOUT, bool BF16>
__device__ __forceinline__ void fast_totals(const CompactStore<BF16>& st, const Geom& G, const KConst<float>& K,
                                            const AoRow& ar, float f[27]) {
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    int64_t e0 = ar.e[1];
    if (LAYOUT) {
      switch (26 - t) {
#define LBMK_CASE(k) case k: e0 = ar.slot0<k, CPLANES>(G); break;
        LBMK_CASE(0) LBMK_CASE(1) LBMK_CASE(2) LBMK_CASE(3) LBMK_CASE(4) LBMK_CASE(5) LBMK_CASE(6)
        LBMK_CASE(7) LBMK_CASE(8) LBMK_CASE(9) LBMK_CASE(10) LBMK_CASE(11) LBMK_CASE(12) LBMK_CASE(13)
        LBMK_CASE(14) LBMK_CASE(15) LBMK_CASE(16) LBMK_CASE(17) LBMK_CASE(18) LBMK_CASE(19) LBMK_CASE(20)
        LBMK_CASE(21) LBMK_CASE(22) LBMK_CASE(23) LBMK_CASE(24) LBMK_CASE(25)
        default: e0 = ar.slot0<26, CPLANES>(G); break;
#undef LBMK_CASE
      }
    }
    f[t] = st.load_at(e0, LAYOUT ? opp_of(t) : t, speed2_of(t), K);
  }
}

// one coordinate of a record tile cell: wrapped across a periodic face, else clamped, with the
// sign that the component of m along that axis takes in the mirror image (-1 beyond the face)
__device__ __forceinline__ int tile_coord(int q, int n, int bc_lo, int bc_hi, float& sgn) {
  sgn = 1.f;
  if (q < 0) {
    if (bc_lo == BC_PERIODIC) return q + n;
    sgn = -1.f;
    return 0;
  }
  if (q >= n) {
    if (bc_hi == BC_PERIODIC && q == n) return 0;
    sgn = -1.f;
    return n - 1;  // also the unused tail cells of a ragged block
  }
  return q;
}

// record tile: cell (cx, cy, cz) holds the record of node (x0-1+cx, y0-1+cy, z0-1+cz), wrapped
// across periodic faces; beyond any other face the record of the face node with the normal
// component of m reversed, which is what a population arriving at the face node from outside
// carries after the specular reflection of a free-slip wall (Sec. IV.A): it left the face node
// itself along the mirrored direction.  (Rows that read the tile are fast rows: in y and z they
// only see cells inside the box, and no-slip x faces exclude them.)  Warp w fills tile rows w,
// w + 8, w + 16; lanes take the columns, lanes 0 and 1 also columns 32 and 33.
template <bool BF16>
__device__ __forceinline__ void fill_record_tile(const CompactStore<BF16>& st, const Geom& G, int x0, int y0,
                                                 int z0, float4* rt, int tid) {
  const int warp = tid >> 5, lane = tid & 31;
  float sa, sb;
  const int xa = tile_coord(x0 - 1 + lane, G.nx, G.bc[0], G.bc[1], sa);
  const int xb = tile_coord(x0 + 31 + lane, G.nx, G.bc[0], G.bc[1], sb);
#pragma unroll
  for (int k = 0; k < (TY * TZ + NWARPS - 1) / NWARPS; ++k) {
    const int row = warp + k * NWARPS;
    if (row < TY * TZ) {
      float sy, sz;
      const int gy = tile_coord(y0 - 1 + row % TY, G.ny, G.bc[2], G.bc[3], sy);
      const int gz = tile_coord(z0 - 1 + row / TY, G.nz, G.bc[4], G.bc[5], sz);
      const float4* rrow = st.rec + snode(G, 0, gy, gz);
      const float4 a = rrow[xa];
      rt[row * TX + lane] = make_float4(a.x, sa * a.y, sy * a.z, sz * a.w);
      if (lane < TX - 32) {
        const float4 b = rrow[xb];
        rt[row * TX + 32 + lane] = make_float4(b.x, sb * b.y, sy * b.z, sz * b.w);
      }
    }
  }
}

// pass 1 (compact): rho and the rebuilt red density of every node -> (rho, phi).  The totals are
// loaded first and the record tile filled while they arrive; on a fast row the value arriving
// along c_t left node x - c_t along c_t (x faces mirrored in the tile), elsewhere the emitter is
// the owner of S(x, opp(t)) and its direction opp(stored direction) (records read directly)
template <bool BF16>
__global__ void __launch_bounds__(NTHREADS, 3) k_density_c(CompactStore<BF16> st, const __grid_constant__ Geom G,
                                                           const __grid_constant__ KConst<float> K, int layout,
                                                           float2* __restrict__ dens, int* __restrict__ flag) {
  __shared__ float4 rt[TILE];
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * BZ;
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
  const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
  const bool active = x < G.nx && y < G.ny && z < G.nz;
  const bool top = on_top(G, z);
  const bool fast = !top && fast_row(G, y, z);
  float f[27];
  if (active && !top) {
    if (fast) {
      AoRow ar;
      ar.init<CPLANES>(G, x, y, z);
      if (!layout) fast_totals<0>(st, G, K, ar, f);
      else fast_totals<1>(st, G, K, ar, f);
    } else {
      NodeMap nm;
      nm.init(G, x, y, z);
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        int64_t node;
        int dir;
        slot_of(nm, layout, t, node, dir);
        f[t] = st.load(node, dir, speed2_of(t), K);
      }
    }
  }
  fill_record_tile(st, G, x0, y0, z0, rt, tid);
  __syncthreads();
  if (!active) return;
  float rho = 0.f, rr = 0.f;
  if (top) {
    const float* tp = G.ctop + ((int64_t)x + (int64_t)G.nx * y) * 64;
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      rr += tp[t];
      rho += tp[t] + tp[32 + t];
    }
  } else if (fast) {
    const int lx = threadIdx.x + 1, ly = threadIdx.y + 1, lz = threadIdx.z + 1;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};  // sum of c_t . m(emitter) per speed class
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      rho += f[t];
      const float4 r = rt[(lx - cx_of(t)) + TX * ((ly - cy_of(t)) + TY * (lz - cz_of(t)))];
      rr = fmaf(r.x, f[t], rr);
      if (t != REST) acc[speed2_of(t)] += cdot_c(t, r.y, r.z, r.w);
    }
#pragma unroll
    for (int s = 1; s < 4; ++s) rr = fmaf(split_coef(s), acc[s], rr);
  } else {
    NodeMap nm;
    nm.init(G, x, y, z);
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      int64_t src;
      int sdir;
      slot_of(nm, 1, t, src, sdir);  // S(x, opp(t)): its owner emitted the value, along opp(sdir)
      rho += f[t];
      rr += red_of(f[t], st.rec[src], opp_of(sdir));
    }
  }
  if (!(rho > 0.f) || !(rho < 1e30f)) atomicOr(flag, 1);
  dens[dnode(G, x, y, z)] = make_float2(rho, (rr + rr - rho) / rho);
}

// pass 2 (compact): gradients + collision + perturbation + recolouring record + streaming of
// the totals (AA pattern); counter protocol as k_collide_stream
template <bool BF16>
__global__ void __launch_bounds__(NTHREADS, 4)
    k_collide_stream_c(CompactStore<BF16> st, const __grid_constant__ Geom G, const __grid_constant__ KConst<float> K,
                       int odd, const float2* __restrict__ dens, long long* __restrict__ counter) {
  __shared__ float2 tile[TILE];
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * BZ;
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
  const bool active = x < G.nx && y < G.ny && z < G.nz;
  const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
  const long long step = counter[odd];
  if (tid == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) counter[odd ^ 1] = step + 1;

  float ft[27];
  const bool fast = fast_row(G, y, z);
  if (active) {
    if (on_top(G, z)) {
      const float* tp = G.ctop + ((int64_t)x + (int64_t)G.nx * y) * 64;
#pragma unroll
      for (int t = 0; t < 27; ++t) ft[t] = tp[t] + tp[32 + t];
    } else if (fast) {
      AoRow ar;
      ar.init<CPLANES>(G, x, y, z);
      if (!odd) {
#pragma unroll
        for (int t = 0; t < 27; ++t) ft[t] = st.load_at(ar.e[1], t, speed2_of(t), K);
      } else {
#pragma unroll
        for (int t = 0; t < 27; ++t) {
          int64_t e0;
          switch (26 - t) {
#define LBMK_CASE(k) case k: e0 = ar.slot0<k, CPLANES>(G); break;
            LBMK_CASE(0) LBMK_CASE(1) LBMK_CASE(2) LBMK_CASE(3) LBMK_CASE(4) LBMK_CASE(5) LBMK_CASE(6)
            LBMK_CASE(7) LBMK_CASE(8) LBMK_CASE(9) LBMK_CASE(10) LBMK_CASE(11) LBMK_CASE(12) LBMK_CASE(13)
            LBMK_CASE(14) LBMK_CASE(15) LBMK_CASE(16) LBMK_CASE(17) LBMK_CASE(18) LBMK_CASE(19) LBMK_CASE(20)
            LBMK_CASE(21) LBMK_CASE(22) LBMK_CASE(23) LBMK_CASE(24) LBMK_CASE(25)
            default: e0 = ar.slot0<26, CPLANES>(G); break;
#undef LBMK_CASE
          }
          ft[t] = st.load_at(e0, opp_of(t), speed2_of(t), K);
        }
      }
    } else {
      NodeMap nm;
      nm.init(G, x, y, z);
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        int64_t node;
        int dir;
        slot_of(nm, odd, t, node, dir);
        ft[t] = st.load(node, dir, speed2_of(t), K);
      }
    }
  }

  // halo tile of (rho, phi), as in k_collide_stream; the Dirichlet inlet nodes carry rho_r0 and
  // phi = 1 (pass 1 stores their true densities, which the macroscopic fields report)
  {
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
        const int cy = gy < G.ny ? gy : G.ny - 1, cz = gz <= tile_zmax(G) ? gz : tile_zmax(G);
        const int64_t rbase = (int64_t)G.nx * ((int64_t)cy + (int64_t)G.ny * cz);
        tile[row * TX + lane] = dens[rbase + cxa];
        if (lane < TX - 32) tile[row * TX + 32 + lane] = dens[rbase + cxb];
      }
    }
    if (G.inflow && z0 == 0) {  // block-uniform: tile planes 0 (z = -1, mirrored onto z = 0) and 1 (z = 0)
      __syncthreads();
      const float rho_r0f = (float)K.rho_r0_d;
      for (int c = tid; c < TX * TY; c += NTHREADS) {
        int gx = wrap_or_clamp(x0 + c % TX - 1, G.nx, G.bc[0], G.bc[1]);
        int gy = wrap_or_clamp(y0 + c / TX - 1, G.ny, G.bc[2], G.bc[3]);
        gx = gx < G.nx ? gx : G.nx - 1;
        gy = gy < G.ny ? gy : G.ny - 1;
        if (is_inlet(G, gx, gy, 0)) {
          tile[c] = make_float2(rho_r0f, 1.0f);
          tile[c + TX * TY] = make_float2(rho_r0f, 1.0f);
        }
      }
    }
  }
  __syncthreads();
  if (!active) return;

  float gphi[3], grho[3];
  const int lx = threadIdx.x + 1, ly = threadIdx.y + 1, lz = threadIdx.z + 1;
  tile_gradients<float>(tile, lx, ly, lz, gphi, grho);
  float f[27];
  float4 record;
  if (is_inlet(G, x, y, z)) {
    inlet_state(K, dnode(G, x, y, z), (int64_t)step, f);
    record = make_float4(1.f, 0.f, 0.f, 0.f);
  } else {
    const float2 c = tile[lx + TX * (ly + TY * lz)];
    const float rho_r = 0.5f * c.x * (1.f + c.y);
    const Recol<float> rc = collide(K, rho_r, ft, gphi, grho, f);
    record = make_float4(rc.frac, rc.cr * rc.n0, rc.cr * rc.n1, rc.cr * rc.n2);
  }
  st.rec[snode(G, x, y, z)] = record;
  if (fast) {
    AoRow ar;
    ar.init<CPLANES>(G, x, y, z);
    if (!odd) {
#pragma unroll
      for (int t = 0; t < 27; ++t) st.store_at(ar.e[1], opp_of(t), speed2_of(t), K, f[t]);
    } else {
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        int64_t e0;
        switch (t) {
#define LBMK_CASE(k) case k: e0 = ar.slot0<k, CPLANES>(G); break;
          LBMK_CASE(0) LBMK_CASE(1) LBMK_CASE(2) LBMK_CASE(3) LBMK_CASE(4) LBMK_CASE(5) LBMK_CASE(6)
          LBMK_CASE(7) LBMK_CASE(8) LBMK_CASE(9) LBMK_CASE(10) LBMK_CASE(11) LBMK_CASE(12) LBMK_CASE(13)
          LBMK_CASE(14) LBMK_CASE(15) LBMK_CASE(16) LBMK_CASE(17) LBMK_CASE(18) LBMK_CASE(19) LBMK_CASE(20)
          LBMK_CASE(21) LBMK_CASE(22) LBMK_CASE(23) LBMK_CASE(24) LBMK_CASE(25)
          default: e0 = ar.slot0<26, CPLANES>(G); break;
#undef LBMK_CASE
        }
        st.store_at(e0, t, speed2_of(t), K, f[t]);
      }
    }
  } else {
    NodeMap nm;
    nm.init(G, x, y, z);
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      int64_t node;
      int dir;
      if (!odd) {
        node = nm.base;
        dir = opp_of(t);
      } else {
        slot_of(nm, 1, 26 - t, node, dir);  // S(x, t)
      }
      st.store(node, dir, speed2_of(t), K, f[t]);
    }
  }
}

// convective outflow (Sec. IV.A) on the compact storage: the node below the top plane is read
// (totals and rebuilt colours), the top plane's per-colour populations live in Geom::ctop only
template <bool BF16>
__global__ void __launch_bounds__(256) k_outflow_c(CompactStore<BF16> st, Geom G,
                                                   const __grid_constant__ KConst<float> K, int layout) {
  const int64_t Pn = (int64_t)G.nx * G.ny;
  const int64_t pp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;  // warp-uniform
  if (pp >= Pn) return;
  const int lane = threadIdx.x & 31;
  const bool act = lane < 27;
  const int t = act ? lane : 0;
  const int x = (int)(pp % G.nx), y = (int)(pp / G.nx);
  NodeMap below;
  below.init(G, x, y, G.nz - 2);
  float fr = 0.f, fb = 0.f;
  if (act) {
    int64_t node, src;
    int dir, sdir;
    slot_of(below, layout, t, node, dir);
    slot_of(below, 1, t, src, sdir);
    const float v = st.load(node, dir, speed2_of(t), K);
    fr = red_of(v, st.rec[src], opp_of(sdir));
    fb = v - fr;
  }
  const float v = fr + fb;
  const float rho = warp_allsum(v);
  const float mz = warp_allsum(cz_of(t) > 0 && act ? v : cz_of(t) < 0 && act ? -v : 0.f);
  float F[3];
  body_force(K, rho, F);
  const float uz = (mz + 0.5f * F[2]) / rho;
  const float lam = uz > 0.f ? uz : 0.f;
  const float inv = 1.f / (1.f + lam);
  if (act) {
    float* tr = G.ctop + pp * 64 + t;
    tr[0] = (tr[0] + lam * fr) * inv;
    tr[32] = (tr[32] + lam * fb) * inv;
  }
}

// initial state: totals of f^k = f^{k(e)}(rho_k, u, alpha_k), Phi = 0, in layout 0; (rho, phi)
// from the given fields; the top plane's per-colour populations into Geom::ctop
template <bool BF16>
__global__ void k_init_c(CompactStore<BF16> st, Geom G, const __grid_constant__ KConst<float> K,
                         const double* __restrict__ rr, const double* __restrict__ rb, const double* __restrict__ u,
                         float2* __restrict__ dens) {
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
    const double fr = r * (vr + poly), fb = b * (vb + poly);
    st.store(sn, t, speed2_of(t), K, (float)(fr + fb));
    if (on_top(G, z)) {
      G.ctop[((int64_t)x + (int64_t)G.nx * y) * 64 + t] = (float)fr;
      G.ctop[((int64_t)x + (int64_t)G.nx * y) * 64 + 32 + t] = (float)fb;
    }
  }
  dens[n] = make_float2((float)(r + b), (float)((r - b) / (r + b)));
}

// rho_r, rho_b, u (Eq. Momentum) into FP64 device buffers (any may be null); rho_r from the
// (rho, phi) field of pass 1 for the current state
template <bool BF16>
__global__ void k_macro_c(CompactStore<BF16> st, Geom G, const __grid_constant__ KConst<float> K, int layout,
                          const float2* __restrict__ dens, double* __restrict__ rr, double* __restrict__ rb,
                          double* __restrict__ u) {
  const int64_t N = (int64_t)G.nx * G.ny * G.nz;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int x = (int)(n % G.nx), y = (int)((n / G.nx) % G.ny), z = (int)(n / ((int64_t)G.nx * G.ny));
  double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, red = 0.0;
  const bool top = on_top(G, z);
  NodeMap nm;
  nm.init(G, x, y, z);
  for (int t = 0; t < 27; ++t) {
    double f;
    if (top) {
      const float* tp = G.ctop + ((int64_t)x + (int64_t)G.nx * y) * 64;
      f = (double)tp[t] + (double)tp[32 + t];
      red += (double)tp[t];
    } else {
      int64_t node;
      int dir;
      slot_of(nm, layout, t, node, dir);
      f = (double)st.load(node, dir, speed2_of(t), K);
    }
    rho += f;
    j[0] += cx_of(t) * f;
    j[1] += cy_of(t) * f;
    j[2] += cz_of(t) * f;
  }
  if (!top) red = 0.5 * rho * (1.0 + (double)dens[n].y);
  double k = 0.0;
  if (K.force_mode == FORCE_BUOYANCY || K.force_mode == FORCE_DISPERSED) k = rho - (double)K.rho_ref;
  else if (K.force_mode == FORCE_UNIFORM) k = 1.0;
  if (rr) rr[n] = red;
  if (rb) rb[n] = rho - red;
  if (u) {
    u[n] = (j[0] + 0.5 * k * (double)K.g[0]) / rho;
    u[N + n] = (j[1] + 0.5 * k * (double)K.g[1]) / rho;
    u[2 * N + n] = (j[2] + 0.5 * k * (double)K.g[2]) / rho;
  }
}

// one direction (paper order) of the canonical FP64 arrays <- storage, colours rebuilt
template <bool BF16>
__global__ void k_get_pop_c(CompactStore<BF16> st, Geom G, const __grid_constant__ KConst<float> K, int layout,
                            int pdir, double* __restrict__ out_r, double* __restrict__ out_b) {
  const int64_t N = (int64_t)G.nx * G.ny * G.nz;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int x = (int)(n % G.nx), y = (int)((n / G.nx) % G.ny), z = (int)(n / ((int64_t)G.nx * G.ny));
  const int t = paper_to_tensor(pdir);
  if (on_top(G, z)) {
    const float* tp = G.ctop + ((int64_t)x + (int64_t)G.nx * y) * 64;
    out_r[n] = tp[t];
    out_b[n] = tp[32 + t];
    return;
  }
  NodeMap nm;
  nm.init(G, x, y, z);
  int64_t node, src;
  int dir, sdir;
  slot_of(nm, layout, t, node, dir);
  slot_of(nm, 1, t, src, sdir);
  const float f = st.load(node, dir, speed2_of(t), K);
  const float fr = red_of(f, st.rec[src], opp_of(sdir));
  out_r[n] = fr;
  out_b[n] = f - fr;
}

// one direction of caller populations -> totals (and the top plane's colours); the colour sums
// per node are accumulated for the (rho, phi) field
template <bool BF16>
__global__ void k_set_pop_c(CompactStore<BF16> st, Geom G, const __grid_constant__ KConst<float> K, int layout,
                            int pdir, const double* __restrict__ in_r, const double* __restrict__ in_b,
                            double* __restrict__ acc_r, double* __restrict__ acc_b) {
  const int64_t N = (int64_t)G.nx * G.ny * G.nz;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int x = (int)(n % G.nx), y = (int)((n / G.nx) % G.ny), z = (int)(n / ((int64_t)G.nx * G.ny));
  const int t = paper_to_tensor(pdir);
  const double r = in_r[n], b = in_b[n];
  acc_r[n] = (pdir == 0 ? 0.0 : acc_r[n]) + r;
  acc_b[n] = (pdir == 0 ? 0.0 : acc_b[n]) + b;
  if (on_top(G, z)) {
    G.ctop[((int64_t)x + (int64_t)G.nx * y) * 64 + t] = (float)r;
    G.ctop[((int64_t)x + (int64_t)G.nx * y) * 64 + 32 + t] = (float)b;
  }
  NodeMap nm;
  nm.init(G, x, y, z);
  int64_t node;
  int dir;
  slot_of(nm, layout, t, node, dir);
  st.store(node, dir, speed2_of(t), K, (float)(r + b));
}

static __global__ void k_dens_from_acc(Geom G, const double* __restrict__ acc_r, const double* __restrict__ acc_b,
                                float2* __restrict__ dens) {
  const int64_t N = (int64_t)G.nx * G.ny * G.nz;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double r = acc_r[n], b = acc_b[n];
  dens[n] = make_float2((float)(r + b), (float)((r - b) / (r + b)));
}

}  // namespace lbmk
