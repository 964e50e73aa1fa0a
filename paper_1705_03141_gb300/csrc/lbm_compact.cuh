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
#include "lbm_tma.cuh"

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
  // by a node's base pointer p1 = A + e1 and a 32-bit element offset (fast rows)
  __device__ __forceinline__ float load_rel(const uint16_t* p1, int rel, int dir, int cls,
                                            const KConst<float>& K) const {
    if (dir == REST) {
      const uint32_t hi = __ldcs(p1 + (rel + REST_HI * 32)), lo = __ldcs(p1 + (rel + REST_LO * 32));
      return __uint_as_float((hi << 16) | lo);
    }
    return K.refB[cls] + dev_to_float(__ldcs(p1 + (rel + dir * 32)));
  }
  __device__ __forceinline__ void store_rel(uint16_t* p1, int rel, int dir, int cls, const KConst<float>& K,
                                            float f) const {
    if (dir == REST) {
      const uint32_t b = __float_as_uint(f);
      __stcs(p1 + (rel + REST_HI * 32), (uint16_t)(b >> 16));
      __stcs(p1 + (rel + REST_LO * 32), (uint16_t)(b & 0xFFFFu));
      return;
    }
    __stcs(p1 + (rel + dir * 32), float_to_dev(f - K.refB[cls]));
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

// red part of a slot: total f, record r of the emitting node, direction j it left along.  Every
// rounding is explicit (no multiply-add contraction left to the compiler), so the value does not
// depend on whether j is known at compile time: the kernels that rebuild the red density on
// different code paths agree bitwise.
__device__ __forceinline__ float red_of(float f, const float4& r, int j) {
  if (j == REST) return __fmul_rn(r.x, f);
  const float cm = __fadd_rn(__fadd_rn(__fmul_rn((float)cx_of(j), r.y), __fmul_rn((float)cy_of(j), r.z)),
                             __fmul_rn((float)cz_of(j), r.w));
  return fmaf(split_coef(speed2_of(j)), cm, __fmul_rn(r.x, f));
}

__device__ __forceinline__ bool on_top(const Geom& G, int z) { return G.ctop != nullptr && z == G.nz - 1; }

// loads of the 27 totals of a node on a fast row: direction t in layout 0 from the node's own
// slot t, in layout 1 from the slot S(x, opp(t))
template <int LAYOUT, bool BF16>
__device__ __forceinline__ void fast_totals(const CompactStore<BF16>& st, const Geom& G, const KConst<float>& K,
                                            const AoRow& ar, float f[27]) {
  const uint16_t* p1 = st.A + ar.e[1];
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    int rel = 0;
    if (LAYOUT) {
      switch (26 - t) {
#define LBMK_CASE(k) case k: rel = ar.rel0<k, CPLANES>(G); break;
        LBMK_CASE(0) LBMK_CASE(1) LBMK_CASE(2) LBMK_CASE(3) LBMK_CASE(4) LBMK_CASE(5) LBMK_CASE(6)
        LBMK_CASE(7) LBMK_CASE(8) LBMK_CASE(9) LBMK_CASE(10) LBMK_CASE(11) LBMK_CASE(12) LBMK_CASE(13)
        LBMK_CASE(14) LBMK_CASE(15) LBMK_CASE(16) LBMK_CASE(17) LBMK_CASE(18) LBMK_CASE(19) LBMK_CASE(20)
        LBMK_CASE(21) LBMK_CASE(22) LBMK_CASE(23) LBMK_CASE(24) LBMK_CASE(25)
        default: rel = ar.rel0<26, CPLANES>(G); break;
#undef LBMK_CASE
      }
    }
    f[t] = st.load_rel(p1, rel, LAYOUT ? opp_of(t) : t, speed2_of(t), K);
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
  const bool top = on_top(G, z);
  const bool fast = !top && fast_row(G, y, z);
  const bool active = x < G.nx && y < G.ny && z < G.nz;
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
      rr = __fadd_rn(rr, red_of(f[t], st.rec[src], opp_of(sdir)));
    }
  }
  if (!(rho > 0.f) || !(rho < 1e30f)) atomicOr(flag, 1);
  dens[dnode(G, x, y, z)] = make_float2(rho, (rr + rr - rho) / rho);
}

// pass 1 (compact), pipelined through the tensor memory accelerator.  The one-block-per-tile pass 1
// above is latency-bound: each block waits for its totals and its record tile, then computes
// briefly.  Here a persistent block of NG consumer groups (8 warps each: one 32 x BY x BZ tile, one
// node per thread) and one producer warp walks over the tiles of the box; the producer copies each
// tile's inputs into a ring of S shared-memory stages while the groups work on earlier tiles, so
// the consumers read shared memory only.  Per tile and step parity, tiled TMA copies of
//   even steps (the node's own slots): one box of the tile's 8 rows of whole 32-node blocks;
//   odd steps (slot S(x, opp(t)) = plane p = opp(t) of node x + c_p): the planes with one c_z form
//     a contiguous run of 9 planes in a block; per c_z one box of that run over the rows
//     y0-1 .. y0+BY (every c_y) and the BZ rows shifted by c_z; plus the tile's own rows of
//     plane 27 (the low half of the rest direction);
//   the record tile (TX x TY x TZ records around the tile);
// and, odd steps, the word the lane at a block edge needs from the neighbouring block in x (the
// last word of plane p for c_p,x = -1, the first for +1; nine planes per side and row), copied
// by the producer lanes with 4-byte asynchronous copies that the stage's barrier also waits for.
// At a reflecting x face the face lane reads plane p -/+ 2 of its own node instead (the mirror of
// AoRow), and the record of the face node with m_x reversed (per-lane offsets and signs).
// Coordinates outside the box read zeros.  Rows that are not fast rows (next to a y or z face, or
// the outflow plane) are left out of the tiles, so no tile waits on global-memory latency: before
// their first tile, all consumer warps of the grid share those rows on the general per-node path
// from global memory, while the producers fill the first stages.  Periodic x faces keep the
// one-block-per-tile kernel for the whole box.
struct DcMaps {
  CUtensorMap rest;  // totals as a 5-d tensor (word, plane, block, y, z + 1): box 32 x 1 x 1 x BY x BZ
  CUtensorMap grp;   // totals as 8-byte words (block, y, z + 1): box 72 x 1 x (BY + 2) x BZ (9 planes)
  CUtensorMap even;  // totals as 8-byte words: box 224 x 1 x BY x BZ (whole blocks of the tile's rows)
  CUtensorMap rec;   // records as floats (4 x, y, z + 1): box 4 TX x TY x TZ (the record tile)
};
constexpr int DC_ROW = 9 * 64;                     // one row of a 9-plane run, bytes
constexpr int DC_GRP = DC_ROW * (BY + 2) * BZ;     // one c_z group box
constexpr int DC_POP = 3 * DC_GRP + BY * BZ * 64;  // odd layout; the even one ([BZ][BY][28][32] words) fits
constexpr int DC_REC = TILE * 16;
constexpr int DC_EDGE = 2 * 9 * BY * BZ * 4;       // [side][plane k][row] 4-byte word pairs
constexpr int DC_STAGE = ((DC_POP + DC_REC + DC_EDGE + 127) / 128) * 128;
static_assert(DC_GRP % 128 == 0 && DC_POP % 128 == 0 && DC_REC % 128 == 0 && DC_POP >= BY * BZ * 1792,
              "TMA destinations on 128-byte boundaries");
__host__ __device__ constexpr uint32_t dc_bytes(int layout) {
  return (layout ? 3 * DC_GRP + BY * BZ * 64 : BY * BZ * 1792) + DC_REC;
}
// pipeline shape: consumer groups per block, stages, blocks per SM
constexpr int DC_NG = 1, DC_S = 3, DC_MINB = 2;
constexpr int DC_THREADS = DC_NG * NTHREADS + 32;
constexpr int DC_SMEM = DC_S * DC_STAGE + 128;

// tile index -> origin (x fastest, then y, then z)
__device__ __forceinline__ void dc_tile(int tile, int ntx, int nty, int& x0, int& y0, int& z0) {
  const int rem = tile / ntx;
  x0 = (tile - rem * ntx) * BX;
  y0 = (rem % nty) * BY;
  z0 = (rem / nty) * BZ;
}

// (rho, phi) of a node that is not on a fast row, from global memory (as pass 1 above)
template <int LAYOUT, bool BF16>
__device__ __forceinline__ void dens_general(const CompactStore<BF16>& st, const Geom& G, const KConst<float>& K,
                                             int x, int y, int z, float2* __restrict__ dens, int* __restrict__ flag) {
  float rho = 0.f, rr = 0.f;
  if (on_top(G, z)) {
    const float* tp = G.ctop + ((int64_t)x + (int64_t)G.nx * y) * 64;
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      rr += tp[t];
      rho += tp[t] + tp[32 + t];
    }
  } else {
    NodeMap nm;
    nm.init(G, x, y, z);
    float f[27];
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      int64_t node;
      int dir;
      slot_of(nm, LAYOUT, t, node, dir);
      f[t] = st.load(node, dir, speed2_of(t), K);
    }
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      int64_t src;
      int sdir;
      slot_of(nm, 1, t, src, sdir);  // S(x, opp(t)): its owner emitted the value, along opp(sdir)
      rho += f[t];
      rr = __fadd_rn(rr, red_of(f[t], st.rec[src], opp_of(sdir)));
    }
  }
  if (!(rho > 0.f) || !(rho < 1e30f)) atomicOr(flag, 1);
  dens[dnode(G, x, y, z)] = make_float2(rho, (rr + rr - rho) / rho);
}

template <bool BF16, int LAYOUT, int NG, int S, int MINB>
__global__ void __launch_bounds__(NG * NTHREADS + 32, MINB)
    k_density_ct(CompactStore<BF16> st, const __grid_constant__ Geom G, const __grid_constant__ KConst<float> K,
                 const __grid_constant__ DcMaps M, float2* __restrict__ dens, int* __restrict__ flag, int ntx,
                 int nty, int ntiles) {
  extern __shared__ __align__(128) unsigned char dc_raw[];
  __shared__ uint64_t full[S], empty[S];
  // stages on 128-byte boundaries; offsetting the shared array itself (not a cast address) keeps
  // every access below a shared-memory access
  unsigned char* const sm = dc_raw + ((128u - (smem_u32(dc_raw) & 127u)) & 127u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NWARPS);
    }
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == NG * NWARPS) {
    // producer warp: the lanes issue the edge-word copies and tie them to the stage's barrier,
    // then lane 0 announces the TMA bytes and lanes 0..4 issue the boxes
    const int XC = G.nxs / 32;
    int j = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
      const int s = j % S;
      if (j >= S && !mbar_wait(&empty[s], ((j / S) & 1) ^ 1)) {
        ok = false;
        break;
      }
      int x0, y0, z0;
      dc_tile(tile, ntx, nty, x0, y0, z0);
      unsigned char* const stg = sm + s * DC_STAGE;
      if (LAYOUT == 1) {
        // edge words: c = side * 72 + k * 8 + row; plane 3k (side 0: word pair 30, 31 of the block
        // before) or 3k + 2 (side 1: words 0, 1 of the block after), row (y0 + ty + c_y, z0 + tz + c_z)
        const int kx = x0 / 32;
        for (int c = lane; c < 2 * 9 * NWARPS; c += 32) {
          const int side = c / 72, k = (c / 8) % 9, r = c % 8;
          const int kb = kx + (side ? 1 : -1);
          const int yy = y0 + r % BY + (k % 3 - 1), zz = z0 + r / BY + (k / 3 - 1);
          if (kb >= 0 && kb < XC && yy >= 0 && yy < G.ny && zz >= -1 && zz <= G.nz) {
            const int64_t blk = (int64_t)kb + (int64_t)XC * ((int64_t)yy + (int64_t)G.ny * (zz + 1));
            const uint16_t* src = st.A + blk * (CPLANES * 32) + (3 * k + 2 * side) * 32 + (side ? 0 : 30);
            cp_async4(stg + DC_POP + DC_REC + c * 4, src);
          }
        }
        cp_async_mbar_arrive(&full[s]);
        __syncwarp();
      }
      if (lane == 0) mbar_arrive_expect_tx(&full[s], dc_bytes(LAYOUT));
      __syncwarp();
      if (lane == 0) {
        tma_load_3d(stg + DC_POP, &M.rec, &full[s], 4 * (x0 - 1), y0 - 1, z0);
      } else if (LAYOUT == 0) {
        if (lane == 1) tma_load_4d(stg, &M.even, &full[s], 0, x0 / 32, y0, z0 + 1);
      } else if (lane <= 3) {
        const int g = lane - 1;  // planes 9g .. 9g+8 (c_z = g - 1), rows y0-1 .. y0+BY, z0+g-1 ..
        tma_load_4d(stg + g * DC_GRP, &M.grp, &full[s], 72 * g, x0 / 32, y0 - 1, z0 + g);
      } else if (lane == 4) {
        tma_load_5d(stg + 3 * DC_GRP, &M.rest, &full[s], 0, REST_LO, x0 / 32, y0, z0 + 1);
      }
    }
    if (!ok) {
      // a wait ran out: report it and let the copies already issued land before the block's
      // shared memory is released (bounded as well)
      if (lane == 0) atomicOr(flag, kFlagTimeout);
      for (int k = j - 1; k >= 0 && k >= j - S; --k) mbar_wait(&full[k % S], (k / S) & 1);
    }
    return;
  }

  // first the rows that are not fast rows, shared among all consumer warps of the grid while the
  // producer fills the first stages: rows y = 0, ny - 1 (every z), then z = 0, nz - 1 (the y
  // between), in 32-node pieces
  {
    const int ntx_ = (G.nx + 31) / 32;
    const int nrow = 2 * G.nz + 2 * (G.ny - 2);
    const int cw = blockIdx.x * (NG * NWARPS) + warp, ncw = gridDim.x * (NG * NWARPS);
    for (int i = cw; i < nrow * ntx_; i += ncw) {
      const int ri = i / ntx_, x = (i - ri * ntx_) * 32 + lane;
      int y, z;
      if (ri < 2 * G.nz) {
        y = (ri & 1) ? G.ny - 1 : 0;
        z = ri >> 1;
      } else {
        z = ((ri - 2 * G.nz) & 1) ? G.nz - 1 : 0;
        y = 1 + ((ri - 2 * G.nz) >> 1);
      }
      if (x < G.nx) dens_general<LAYOUT>(st, G, K, x, y, z, dens, flag);
    }
  }

  // consumer group grp takes the block's tiles grp, grp + NG, ...; warp w of a group is row
  // (w % BY, w / BY) of the tile
  const int grp = warp / NWARPS, row = warp % NWARPS;
  const int ty = row % BY, tz = row / BY;
  const int lx = lane + 1, ly = ty + 1, lz = tz + 1;
  int j = grp;
  for (int tile = blockIdx.x + grp * gridDim.x; tile < ntiles; tile += NG * gridDim.x, j += NG) {
    const int s = j % S;
    if (!mbar_wait(&full[s], (j / S) & 1)) {
      if (lane == 0) atomicOr(flag, kFlagTimeout);
      break;
    }
    int x0, y0, z0;
    dc_tile(tile, ntx, nty, x0, y0, z0);
    const int x = x0 + lane, y = y0 + ty, z = z0 + tz;
    const unsigned char* const stg = sm + s * DC_STAGE;
    const float4* const rt = reinterpret_cast<const float4*>(stg + DC_POP);
    if (x < G.nx && y < G.ny && z < G.nz && !on_top(G, z) && fast_row(G, y, z)) {
      // mirror x faces: the face lane's emitter beyond the face is the face node itself
      const bool mlo = x == 0, mhi = x == G.nx - 1;
      float f[27];
      if (LAYOUT == 0) {
        const unsigned char* const b0 = stg + row * 1792 + lane * 2;
#pragma unroll
        for (int t = 0; t < 27; ++t) {
          if (t == REST) {
            const uint32_t hi = *reinterpret_cast<const uint16_t*>(b0 + REST_HI * 64);
            const uint32_t lo = *reinterpret_cast<const uint16_t*>(b0 + REST_LO * 64);
            f[t] = __uint_as_float((hi << 16) | lo);
          } else {
            f[t] = K.refB[speed2_of(t)] +
                   CompactStore<BF16>::dev_to_float(*reinterpret_cast<const uint16_t*>(b0 + t * 64));
          }
        }
      } else {
        // word x - x0 + c_p,x of a group row; at the block edges the edge word instead (a
        // neighbouring block) or, at a mirror face, plane p -/+ 2 of the lane's own node
        const unsigned char* const r1 = stg + (tz * (BY + 2) + ty + 1) * DC_ROW;
        const unsigned char* const e1 = stg + DC_POP + DC_REC + row * 4;
        const bool em = lane == 0 && !mlo, ep = lane == 31 && !mhi;  // read the edge words
        const unsigned char* const bm = mlo ? r1 + lane * 2 + 128 : r1 + (lane > 0 ? lane - 1 : 0) * 2;
        const unsigned char* const bz = r1 + lane * 2;
        const unsigned char* const bp = mhi ? r1 + lane * 2 - 128 : r1 + (lane < 31 ? lane + 1 : 31) * 2;
#pragma unroll
        for (int t = 0; t < 27; ++t) {
          const int p = opp_of(t), g = cz_of(p) + 1;
          const int go = g * DC_GRP + cy_of(p) * DC_ROW + (p - 9 * g) * 64;  // plane p's offset in a row
          if (t == REST) {
            const uint32_t hi = *reinterpret_cast<const uint16_t*>(bz + go);
            const uint32_t lo = *reinterpret_cast<const uint16_t*>(stg + 3 * DC_GRP + row * 64 + lane * 2);
            f[t] = __uint_as_float((hi << 16) | lo);
          } else {
            const unsigned char* a;
            if (cx_of(p) < 0) a = em ? e1 + (p / 3) * 32 + 2 : bm + go;
            else if (cx_of(p) > 0) a = ep ? e1 + 288 + ((p - 2) / 3) * 32 : bp + go;
            else a = bz + go;
            f[t] = K.refB[speed2_of(t)] + CompactStore<BF16>::dev_to_float(*reinterpret_cast<const uint16_t*>(a));
          }
        }
      }
      // records: emitter x - c_t; beyond a mirror face the face node's own record (one column
      // over) with m_x reversed
      const float4* const rc = rt + lx + TX * (ly + TY * lz);
      const float4* const rlo = rc + (mlo ? 1 : 0);  // directions with c_x = +1
      const float4* const rhi = rc - (mhi ? 1 : 0);  // directions with c_x = -1
      const float klo = mlo ? -1.f : 1.f, khi = mhi ? 1.f : -1.f;  // factor of m_x in c_t . m
      float rho = 0.f, rr = 0.f;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};  // sum of c_t . m(emitter) per speed class
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        rho += f[t];
        const float4* const base = cx_of(t) > 0 ? rlo : (cx_of(t) < 0 ? rhi : rc);
        const float4 r = base[-cx_of(t) - TX * (cy_of(t) + TY * cz_of(t))];
        rr = fmaf(r.x, f[t], rr);
        if (t != REST) {
          // c_t . m by signed additions in the order of cdot_c (a product with +-1 is exact)
          float cm = -0.0f;
          if (cx_of(t) > 0) cm = fmaf(klo, r.y, cm);
          if (cx_of(t) < 0) cm = fmaf(khi, r.y, cm);
          if (cy_of(t) > 0) cm += r.z;
          if (cy_of(t) < 0) cm -= r.z;
          if (cz_of(t) > 0) cm += r.w;
          if (cz_of(t) < 0) cm -= r.w;
          acc[speed2_of(t)] += cm;
        }
      }
#pragma unroll
      for (int c = 1; c < 4; ++c) rr = fmaf(split_coef(c), acc[c], rr);
      if (!(rho > 0.f) || !(rho < 1e30f)) atomicOr(flag, 1);
      dens[dnode(G, x, y, z)] = make_float2(rho, (rr + rr - rho) / rho);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);  // the stage goes back to the producer
  }
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
      if (!odd) fast_totals<0>(st, G, K, ar, ft);
      else fast_totals<1>(st, G, K, ar, ft);
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
    uint16_t* p1 = st.A + ar.e[1];
    if (!odd) {
#pragma unroll
      for (int t = 0; t < 27; ++t) st.store_rel(p1, 0, opp_of(t), speed2_of(t), K, f[t]);
    } else {
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        int rel;
        switch (t) {
#define LBMK_CASE(k) case k: rel = ar.rel0<k, CPLANES>(G); break;
          LBMK_CASE(0) LBMK_CASE(1) LBMK_CASE(2) LBMK_CASE(3) LBMK_CASE(4) LBMK_CASE(5) LBMK_CASE(6)
          LBMK_CASE(7) LBMK_CASE(8) LBMK_CASE(9) LBMK_CASE(10) LBMK_CASE(11) LBMK_CASE(12) LBMK_CASE(13)
          LBMK_CASE(14) LBMK_CASE(15) LBMK_CASE(16) LBMK_CASE(17) LBMK_CASE(18) LBMK_CASE(19) LBMK_CASE(20)
          LBMK_CASE(21) LBMK_CASE(22) LBMK_CASE(23) LBMK_CASE(24) LBMK_CASE(25)
          default: rel = ar.rel0<26, CPLANES>(G); break;
#undef LBMK_CASE
        }
        st.store_rel(p1, rel, t, speed2_of(t), K, f[t]);
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
#pragma unroll
  for (int t = 0; t < 27; ++t) {  // the lattice constants fold at compile time
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
