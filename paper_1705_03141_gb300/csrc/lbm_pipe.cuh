// Collide-stream pass for packed storage with the populations staged by TMA (variant 5).
//
// The one-node kernel k_collide_stream is bound by instruction issue: its warps wait on the 27
// global loads of their node, and on odd steps each load and store also pays for the slot's
// address.  Here persistent blocks walk over the box's interior tiles (32 x BY x BZ nodes whose
// rows are all fast rows); per block, one producer warp copies a tile's population words and its
// (rho, phi) halo into a shared-memory stage with tiled cp.async.bulk.tensor copies, while the
// 8 consumer warps compute the tile before it.  Consumers read their populations from shared
// memory at compile-time offsets from one per-thread address, release the stage once the
// populations and gradients are in registers, then collide and store to global memory as the
// one-node kernel does.  The tiles that touch a y or z face (rows next to walls, the inlet and
// the outflow plane) are left to the one-node kernel, launched over just those tiles.
//
// Stage layout (one tile; every TMA destination on a 128-byte boundary):
//   even step  [BZ][BY][27 planes][32 words]: the tile's own rows, slot (x, t) of node x;
//   odd step   slot S(x, opp(t)) is plane T = opp(t) of node x + c_T: for each row group
//              G = (c_y + 1) + 3 (c_z + 1) (planes 3G .. 3G+2, c_x = -1, 0, 1) one box
//              [BZ][BY][3][32] of the rows y0+c_y .. y0+c_y+BY-1, z0+c_z .. z0+c_z+BZ-1, each
//              followed by a 128-byte pad that holds the words the block-edge lanes need from
//              the neighbouring 32-node blocks ([side][tile row], plane 3G or 3G+2; 4-byte
//              cp.async tied to the stage's barrier), so that every lane finds the word of
//              direction t at one compile-time offset from its own base address; a lane on a
//              reflecting x face reads plane T -/+ 2 of its own node instead (the mirror of AoRow);
//   both       the (rho, phi) halo tile, 36 x TY x TZ cells as in k_collide_stream.
// Every wait is bounded (mbar_wait_sleep: waiting warps sleep in the try-wait instead of spinning
// on it, which leaves the issue slots to the other block of the SM): one that runs out raises kFlagTimeout, which
// lbm_synchronize reports as LBM_ETIMEOUT, and the producer lets its issued copies land first.
#pragma once
#include "lbm_kernels.cuh"
#include "lbm_tma.cuh"

namespace lbmk {

struct TpMaps {
  CUtensorMap even;  // packed words (word 32, plane 27, block, y, z + 1): box 32 x 27 x 1 x BY x BZ
  CUtensorMap grp;   // the same tensor: box 32 x 3 x 1 x BY x BZ (one row group)
  CUtensorMap dens;  // (rho, phi) cells (x, y, z + 1): box 36 x TY x TZ
};

constexpr int TP_ROW = 27 * 128;                  // one row of a tile, all planes (even), bytes
constexpr int TP_GROW = 3 * 128;                  // one row of a row group (odd)
constexpr int TP_GRP = TP_GROW * BY * BZ;         // one row-group box
constexpr int TP_GS = TP_GRP + 128;               // a row-group box and its edge-word pad (odd)
constexpr int TP_POP = 9 * TP_GS;                 // populations of a stage (the even box fits)
constexpr int TP_DOFF = TP_POP;                   // the (rho, phi) tile
constexpr int TP_DENS = BlkDefault::TILET * 8;
constexpr int TP_STAGE = ((TP_DOFF + TP_DENS + 127) / 128) * 128;
static_assert(TP_GRP % 128 == 0 && TP_POP % 128 == 0 && TP_POP >= BY * BZ * TP_ROW && 2 * NWARPS * 4 <= 128,
              "stage layout");
constexpr int TP_S = 2, TP_MINB = 2;  // stages per block, blocks per SM (96 registers, no spills)
constexpr int TP_THREADS = NTHREADS + 32;
constexpr int TP_SMEM = TP_S * TP_STAGE + 128;
__host__ __device__ constexpr uint32_t tp_bytes() { return (uint32_t)(BY * BZ * TP_ROW) + (uint32_t)TP_DENS; }

template <bool BF16, int ODD>
__global__ void __launch_bounds__(TP_THREADS, TP_MINB)
    k_collide_stream_tp(PackedStore<BF16> st, const __grid_constant__ Geom G, const __grid_constant__ KConst<float> K,
                        const __grid_constant__ TpMaps M, const TileSplit ts, int* __restrict__ flag) {
  using B = BlkDefault;
  using Store = PackedStore<BF16>;
  extern __shared__ __align__(128) unsigned char tp_raw[];
  __shared__ uint64_t full[TP_S], empty[TP_S];
  __shared__ int4 origin[TP_S];  // the stage's tile: x0, y0, z0, in-box columns (written by the producer)
  unsigned char* const sm = tp_raw + ((128u - (smem_u32(tp_raw) & 127u)) & 127u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = ts.interior();
  if (tid == 0) {
    for (int s = 0; s < TP_S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NWARPS);
      origin[s] = make_int4(0, 0, 0, (B::TXT - 1) << 8);  // a valid tile even for a wait that runs out
    }
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == NWARPS) {
    // producer: the lanes issue the edge-word copies (odd steps) and tie them to the stage's
    // barrier, lane 0 announces the TMA bytes, lanes 0..1 (even) or 0..9 (odd) issue the boxes
    const int XC = G.nxs / 32;
    int j = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
      const int s = j % TP_S;
      if (j >= TP_S && !mbar_wait_sleep(&empty[s], ((j / TP_S) & 1) ^ 1)) {
        ok = false;
        break;
      }
      int x0, y0, z0;
      ts.interior_tile(tile, BY, BZ, x0, y0, z0);
      unsigned char* const stg = sm + s * TP_STAGE;
      if (ODD) {
        // c = side * 72 + k * 8 + r: plane T = 3k (side 0: word 31 of the block before) or
        // 3k + 2 (side 1: word 0 of the block after), tile row r, source row shifted by c_T
        const int kx = x0 / 32;
        for (int c = lane; c < 2 * 9 * NWARPS; c += 32) {
          const int side = c / 72, k = (c / 8) % 9, r = c % 8;
          const int kb = kx + (side ? 1 : -1);
          const int yy = y0 + r % BY + (k % 3 - 1), zz = z0 + r / BY + (k / 3 - 1);
          if (kb >= 0 && kb < XC) {  // interior tiles: yy, zz lie inside the box
            const int64_t blk = (int64_t)kb + (int64_t)XC * ((int64_t)yy + (int64_t)G.ny * (zz + 1));
            const uint32_t* src = st.A + blk * (27 * 32) + (3 * k + 2 * side) * 32 + (side ? 0 : 31);
            cp_async4(stg + k * TP_GS + TP_GRP + side * 32 + r * 4, src);  // the pad after box k
          }
        }
        cp_async_mbar_arrive(&full[s]);
        __syncwarp();
      }
      if (lane == 0) {
        // in-box columns of the (rho, phi) tile (interior tiles cross no y or z face): cx0 | cx1 << 8
        TileRange tr;
        tr.init<BlkDefault>(G, x0, y0, z0);
        origin[s] = make_int4(x0, y0, z0, tr.cx0 | (tr.cx1 << 8));  // released by the arrive below
        mbar_arrive_expect_tx(&full[s], tp_bytes());
      }
      __syncwarp();
      if (lane == 0) {
        tma_load_3d(stg + TP_DOFF, &M.dens, &full[s], x0 - 2, y0 - 1, z0);  // tensor plane z0 is z = z0 - 1
      } else if (!ODD) {
        if (lane == 1) tma_load_5d(stg, &M.even, &full[s], 0, 0, x0 / 32, y0, z0 + 1);
      } else if (lane <= 9) {
        const int g = lane - 1;  // planes 3g .. 3g+2: rows y0 + c_y .., z0 + c_z .. (tensor z + 1)
        tma_load_5d(stg + g * TP_GS, &M.grp, &full[s], 0, 3 * g, x0 / 32, y0 + g % 3 - 1, z0 + g / 3);
      }
    }
    if (!ok) {
      if (lane == 0) atomicOr(flag, kFlagTimeout);
      for (int k = j - 1; k >= 0 && k >= j - TP_S; --k) mbar_wait(&full[k % TP_S], (k / TP_S) & 1);
    }
    return;
  }

  // consumers: warp w is tile row (w % BY, w / BY)
  const int row = warp, ty = row % BY, tz = row / BY;
  int j = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
    const int s = j % TP_S;
    bool ok = mbar_wait_sleep(&full[s], (j / TP_S) & 1);
    if (!ok) {
      if (lane == 0) atomicOr(flag, kFlagTimeout);
    }
    const int4 o = origin[s];  // the producer's tile origin (no divisions here)
    const int x0 = o.x, y0 = o.y, z0 = o.z;
    const int x = x0 + lane, y = y0 + ty, z = z0 + tz;
    unsigned char* const stg = sm + s * TP_STAGE;
    float2* const dt = reinterpret_cast<float2*>(stg + TP_DOFF);
    // mirror ghosts of the x faces in the (rho, phi) tile (interior tiles cross no y or z face)
    TileRange tr;
    tr.cx0 = o.w & 0xFF;
    tr.cx1 = o.w >> 8;
    tr.cy0 = 0;
    tr.cy1 = B::TY - 1;
    tr.cz0 = 0;
    tr.cz1 = B::TZ - 1;
    if (tr.clamps<B>()) {
      tile_clamp_fix<B>(dt, tr, tid);
      fence_proxy_async();  // these writes land before the stage's next TMA copy
      named_sync(NTHREADS);
    }
    const bool act = x < G.nx;
    float rho_r = 0.f, ft[27], gphi[3], grho[3];
    if (act) {
      float acc = 0.f;
      if (!ODD) {
        const unsigned char* const b0 = stg + row * TP_ROW + lane * 4;
#pragma unroll
        for (int t = 0; t < 27; ++t) {
          const uint32_t w = *reinterpret_cast<const uint32_t*>(b0 + t * 128);
          ft[t] = Store::decode_red(w, K.refB[speed2_of(t)], t == REST ? K.dref[0] : 0.0f, acc);
        }
      } else {
        // word lane + c_T,x of a group row: one base address per c_x; the block-edge lanes'
        // bases point into the pads (side 0 holds plane 3G, side 1 plane 3G + 2), and at a
        // reflecting x face to plane T -/+ 2 of the lane's own node
        const bool mlo = x == 0, mhi = x == G.nx - 1;
        const unsigned char* const r1 = stg + row * TP_GROW;
        const unsigned char* const bm =
            mlo ? r1 + lane * 4 + 256 : (lane == 0 ? stg + TP_GRP + row * 4 : r1 + (lane - 1) * 4);
        const unsigned char* const bz = r1 + lane * 4;
        const unsigned char* const bp =
            mhi ? r1 + lane * 4 - 256 : (lane == 31 ? stg + TP_GRP + 32 + row * 4 - 256 : r1 + (lane + 1) * 4);
#pragma unroll
        for (int t = 0; t < 27; ++t) {
          const int T = opp_of(t), g = T / 3;
          const int go = g * TP_GS + (T - 3 * g) * 128;  // plane T in the node's row of its group box
          const unsigned char* const a = (cx_of(T) < 0 ? bm : (cx_of(T) > 0 ? bp : bz)) + go;
          ft[t] = Store::decode_red(*reinterpret_cast<const uint32_t*>(a), K.refB[speed2_of(t)],
                                    t == REST ? K.dref[0] : 0.0f, acc);
        }
      }
      rho_r = Store::red_finish(acc);
      tile_gradients<float, float2, B::TXT, B::TY>(dt, lane + 2, ty + 1, tz + 1, gphi, grho);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);  // the populations and gradients are in registers
    if (act && ok) {
      float f[27];
      const Recol<float> rc = collide(K, rho_r, ft, gphi, grho, f);
      const bool recol = __any_sync(__activemask(), any_(rc.has_n));
      NodeMap nm;
      AoRow ar;
      ar.init<27>(G, x, y, z);
      if (recol) EmitLoop<0, Store, float, true, true, false, ODD, B::BY, B::TX>::run(st, K, G, nm, ar, ODD != 0, f, rc, nullptr, FusedIO{}, x, y, z);
      else EmitLoop<0, Store, float, true, false, false, ODD, B::BY, B::TX>::run(st, K, G, nm, ar, ODD != 0, f, rc, nullptr, FusedIO{}, x, y, z);
    }
  }
}

}  // namespace lbmk
