// Jet-trajectory surrogate behind include/lbm_mlp.h: a multilayer perceptron
// trained and evaluated on the device.  Matrix products run on the tensor
// cores with bfloat16 operands and FP32 accumulation (mma.sync m16n8k16: the
// products are at most 4096 x 4096 x 256, far too small to need the larger
// asynchronous tensor-core pipeline); epilogues fuse bias, SiLU and its
// derivative; every reduction has a fixed order, so results are reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/lbm_mlp.h"

namespace {

constexpr int TM = 64, TN = 64, TK = 32, GEMM_THREADS = 128;
constexpr int SK = TK + 8;  // padded shared row (bf16): conflict-free fragment loads
constexpr int KSPLIT = 256;  // batch rows per split of a weight-gradient product

enum { EPI_SILU = 0, EPI_LINEAR = 1, EPI_DSILU = 2, EPI_PARTIAL = 3 };

// C(m, n) = sum_k A(m, k) B(n, k); A(m, k) = A[m sAm + k sAk], B(n, k) = B[n sBn + k sBk]
struct GemmArgs {
  const __nv_bfloat16* A;
  long long sAm, sAk;
  const __nv_bfloat16* B;
  long long sBn, sBk;
  int M, N, K;
  int kps;            // K range per blockIdx.z (multiple of TK)
  const float* bias;  // EPI_SILU, EPI_LINEAR
  float* out;         // SILU: z; LINEAR: y; DSILU: dz; PARTIAL: [split][M][N]
  long long ldo;
  __nv_bfloat16* outb;  // SILU: silu(z); DSILU: dz
  long long ldb;
  const float* zsave;  // DSILU: pre-activations
  long long ldz;
};

__device__ __forceinline__ float sigmoid_(float z) { return 1.0f / (1.0f + expf(-z)); }

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// stage a ROWS x TK tile X(r, k) = P[(r0 + r) sr + (k0 + k) sk] (zero outside rows < R, k < kend)
template <int ROWS>
__device__ __forceinline__ void stage(__nv_bfloat16* S, const __nv_bfloat16* P, long long sr, long long sk, int r0,
                                      int R, int k0, int kend) {
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  for (int e = threadIdx.x; e < ROWS * TK; e += GEMM_THREADS) {
    int r, c;
    if (sk == 1) {  // consecutive threads along the contiguous index
      r = e / TK;
      c = e % TK;
    } else {
      c = e / ROWS;
      r = e % ROWS;
    }
    const int gr = r0 + r, gk = k0 + c;
    S[r * SK + c] = (gr < R && gk < kend) ? P[gr * sr + gk * sk] : zero;
  }
}

template <int EPI>
__global__ void __launch_bounds__(GEMM_THREADS) k_gemm(const GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 As[TM * SK];
  __shared__ __align__(16) __nv_bfloat16 Bs[TN * SK];
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int kbeg = blockIdx.z * g.kps;
  const int kend = min(g.K, kbeg + g.kps);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gid = lane >> 2, tig = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.0f;

  for (int k0 = kbeg; k0 < kend; k0 += TK) {
    stage<TM>(As, g.A, g.sAm, g.sAk, m0, g.M, k0, kend);
    stage<TN>(Bs, g.B, g.sBn, g.sBk, n0, g.N, k0, kend);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; kk += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const __nv_bfloat16* p = As + (wm + i * 16 + gid) * SK + kk + 2 * tig;
        a[i][0] = ld_pair(p);
        a[i][1] = ld_pair(p + 8 * SK);
        a[i][2] = ld_pair(p + 8);
        a[i][3] = ld_pair(p + 8 * SK + 8);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const __nv_bfloat16* p = Bs + (wn + j * 8 + gid) * SK + kk + 2 * tig;
        b[j][0] = ld_pair(p);
        b[j][1] = ld_pair(p + 8);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int m = m0 + wm + i * 16 + gid + (c >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + 2 * tig + (c & 1);
        if (m >= g.M || n >= g.N) continue;
        const float v = acc[i][j][c];
        if constexpr (EPI == EPI_SILU) {
          const float z = v + g.bias[n];
          g.out[m * g.ldo + n] = z;
          g.outb[m * g.ldb + n] = __float2bfloat16(z * sigmoid_(z));
        } else if constexpr (EPI == EPI_LINEAR) {
          g.out[m * g.ldo + n] = v + g.bias[n];
        } else if constexpr (EPI == EPI_DSILU) {
          const float z = g.zsave[m * g.ldz + n];
          const float s = sigmoid_(z);
          const float d = v * s * (1.0f + z * (1.0f - s));
          g.out[m * g.ldo + n] = d;
          g.outb[m * g.ldb + n] = __float2bfloat16(d);
        } else {
          g.out[((long long)blockIdx.z * g.M + m) * g.N + n] = v;
        }
      }
}

__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16(x[i]);
}

// per row: squared error of the positions and cross-entropy of the logits, and dL/dy
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ target, const int* __restrict__ label,
                       int B, int n_pos, int n_cls, float w_pos, float w_cls, float* __restrict__ dy,
                       __nv_bfloat16* __restrict__ dyb, float* __restrict__ row_loss, int* __restrict__ bad) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int n_out = n_pos + n_cls;
  const float* yr = y + (long long)b * n_out;
  float* dr = dy + (long long)b * n_out;
  __nv_bfloat16* dbr = dyb + (long long)b * n_out;
  float lp = 0.0f;
  for (int k = 0; k < n_pos; ++k) {
    const float d = yr[k] - target[(long long)b * n_pos + k];
    lp += d * d;
    dr[k] = w_pos * 2.0f * d / (float)(B * n_pos);
  }
  float lc = 0.0f;
  if (n_cls > 0) {
    int lab = label[b];
    if (lab < 0 || lab >= n_cls) {
      atomicOr(bad, 1);
      lab = 0;
    }
    float mx = yr[n_pos];
    for (int k = 1; k < n_cls; ++k) mx = fmaxf(mx, yr[n_pos + k]);
    float se = 0.0f;
    for (int k = 0; k < n_cls; ++k) se += expf(yr[n_pos + k] - mx);
    lc = logf(se) - (yr[n_pos + lab] - mx);
    for (int k = 0; k < n_cls; ++k) {
      const float p = expf(yr[n_pos + k] - mx) / se;
      dr[n_pos + k] = w_cls * (p - (k == lab ? 1.0f : 0.0f)) / (float)B;
    }
  }
  for (int k = 0; k < n_out; ++k) dbr[k] = __float2bfloat16(dr[k]);
  row_loss[b] = (n_pos > 0 ? w_pos * lp / (float)(B * n_pos) : 0.0f) + w_cls * lc / (float)B;
}

// fixed-order sum of n values by one block of 256 threads
__global__ void k_sum(const float* __restrict__ v, int n, float* __restrict__ out) {
  __shared__ float s[256];
  float a = 0.0f;
  for (int i = threadIdx.x; i < n; i += 256) a += v[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// out[n] = sum_b g[b][n] (bias gradients), one thread per column, fixed order
__global__ void k_colsum(const float* __restrict__ g, int B, int N, float* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float a = 0.0f;
  for (int b = 0; b < B; ++b) a += g[(long long)b * N + n];
  out[n] = a;
}

// out[e] = sum_s part[s][e], fixed order
__global__ void k_reduce_splits(const float* __restrict__ part, int splits, long long n, float* __restrict__ out) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  float a = 0.0f;
  for (int s = 0; s < splits; ++s) a += part[s * n + e];
  out[e] = a;
}

// Adam with bias correction; refreshes the bfloat16 copy of the parameters
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ pb, long long n, float lr, float c1,
                       float c2) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
  p[i] = pi;
  pb[i] = __float2bfloat16(pi);
}

bool is_device_ptr(const void* ptr) {
  if (!ptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct lbm_mlp {
  int n_in, width, depth, n_pos, n_cls, n_out, max_batch;
  cudaStream_t stream;
  std::vector<int> fan_in, fan_out;  // per layer
  std::vector<size_t> w_off, b_off;  // flat offsets
  size_t P;
  long long step;
  char* mem;
  float *p, *g, *m, *v;          // parameters, gradient, Adam moments (flat FP32)
  __nv_bfloat16* pb;             // bfloat16 copy of the parameters
  float* x32;                    // staged input [max_batch][n_in]
  __nv_bfloat16* h[9];           // layer inputs: h[0] = x, h[l] = silu(z_l), bf16
  float* z[9];                   // pre-activations z_l, l = 1..depth (FP32)
  float* y;                      // output [max_batch][n_out]
  float *d32[2];                 // backward: dL/dz (FP32), ping-pong
  __nv_bfloat16* d16[2];         // backward: dL/dz (bf16)
  float* part;                   // weight-gradient split partials
  float *tgt, *row_loss, *loss;  // staged targets, per-row loss, total
  int *lab, *bad;
};

namespace {

template <int EPI>
cudaError_t gemm(const GemmArgs& a, int splits, cudaStream_t s) {
  dim3 grid((unsigned)((a.N + TN - 1) / TN), (unsigned)((a.M + TM - 1) / TM), (unsigned)splits);
  k_gemm<EPI><<<grid, GEMM_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

GemmArgs args(const __nv_bfloat16* A, long long sAm, long long sAk, const __nv_bfloat16* B, long long sBn,
              long long sBk, int M, int N, int K) {
  GemmArgs a;
  memset(&a, 0, sizeof a);
  a.A = A;
  a.sAm = sAm;
  a.sAk = sAk;
  a.B = B;
  a.sBn = sBn;
  a.sBk = sBk;
  a.M = M;
  a.N = N;
  a.K = K;
  a.kps = (K + TK - 1) / TK * TK;
  return a;
}

#define MLP_CUDA(call)                              \
  do {                                              \
    if ((call) != cudaSuccess) {                    \
      cudaGetLastError();                           \
      return LBM_ECUDA;                             \
    }                                               \
  } while (0)

// forward pass of `batch` rows already staged in m->x32
lbm_status forward(lbm_mlp* m, int batch) {
  MLP_CUDA((k_to_bf16<<<blocks((long long)batch * m->n_in, 256), 256, 0, m->stream>>>(m->x32, m->h[0],
                                                                                     (long long)batch * m->n_in),
            cudaGetLastError()));
  const int L = m->depth + 1;
  for (int l = 0; l < L; ++l) {
    const int K = m->fan_in[l], N = m->fan_out[l];
    GemmArgs a = args(m->h[l], K, 1, m->pb + m->w_off[l], K, 1, batch, N, K);
    a.bias = m->p + m->b_off[l];
    if (l < L - 1) {
      a.out = m->z[l + 1];
      a.ldo = N;
      a.outb = m->h[l + 1];
      a.ldb = N;
      MLP_CUDA(gemm<EPI_SILU>(a, 1, m->stream));
    } else {
      a.out = m->y;
      a.ldo = N;
      MLP_CUDA(gemm<EPI_LINEAR>(a, 1, m->stream));
    }
  }
  return LBM_OK;
}

// loss and gradient (into m->g) of `batch` rows staged in x32 / tgt / lab
lbm_status backward(lbm_mlp* m, int batch, float w_pos, float w_cls) {
  lbm_status st = forward(m, batch);
  if (st != LBM_OK) return st;
  const int L = m->depth + 1;
  MLP_CUDA(cudaMemsetAsync(m->bad, 0, sizeof(int), m->stream));
  k_loss<<<blocks(batch, 128), 128, 0, m->stream>>>(m->y, m->tgt, m->lab, batch, m->n_pos, m->n_cls, w_pos, w_cls,
                                                     m->d32[0], m->d16[0], m->row_loss, m->bad);
  MLP_CUDA(cudaGetLastError());
  k_sum<<<1, 256, 0, m->stream>>>(m->row_loss, batch, m->loss);
  MLP_CUDA(cudaGetLastError());
  int cur = 0;
  for (int l = L - 1; l >= 0; --l) {
    const int K = m->fan_in[l], N = m->fan_out[l];
    // dW_l(o, i) = sum_b g(b, o) h_{l-1}(b, i): split over the batch, reduced in a fixed order
    const int splits = (batch + KSPLIT - 1) / KSPLIT;
    GemmArgs a = args(m->d16[cur], 1, N, m->h[l], 1, K, N, K, batch);
    a.kps = KSPLIT;
    a.out = m->part;
    MLP_CUDA(gemm<EPI_PARTIAL>(a, splits, m->stream));
    k_reduce_splits<<<blocks((long long)N * K, 256), 256, 0, m->stream>>>(m->part, splits, (long long)N * K,
                                                                         m->g + m->w_off[l]);
    MLP_CUDA(cudaGetLastError());
    k_colsum<<<blocks(N, 128), 128, 0, m->stream>>>(m->d32[cur], batch, N, m->g + m->b_off[l]);
    MLP_CUDA(cudaGetLastError());
    if (l > 0) {
      // dL/dz_{l-1}(b, i) = sum_o g(b, o) W_l(o, i) * silu'(z_{l-1}(b, i))
      GemmArgs d = args(m->d16[cur], N, 1, m->pb + m->w_off[l], 1, K, batch, K, N);
      d.out = m->d32[cur ^ 1];
      d.ldo = K;
      d.outb = m->d16[cur ^ 1];
      d.ldb = K;
      d.zsave = m->z[l];
      d.ldz = K;
      MLP_CUDA(gemm<EPI_DSILU>(d, 1, m->stream));
      cur ^= 1;
    }
  }
  return LBM_OK;
}

lbm_status stage_inputs(lbm_mlp* m, const float* x, const float* target, const int* label, int batch) {
  const cudaMemcpyKind kx = is_device_ptr(x) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  MLP_CUDA(cudaMemcpyAsync(m->x32, x, sizeof(float) * batch * m->n_in, kx, m->stream));
  if (target && m->n_pos > 0) {
    const cudaMemcpyKind kt = is_device_ptr(target) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    MLP_CUDA(cudaMemcpyAsync(m->tgt, target, sizeof(float) * batch * m->n_pos, kt, m->stream));
  }
  if (label && m->n_cls > 0) {
    const cudaMemcpyKind kl = is_device_ptr(label) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    MLP_CUDA(cudaMemcpyAsync(m->lab, label, sizeof(int) * batch, kl, m->stream));
  }
  return LBM_OK;
}

lbm_status copy_out(lbm_mlp* m, void* dst, const void* src, size_t bytes) {
  const cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  MLP_CUDA(cudaMemcpyAsync(dst, src, bytes, k, m->stream));
  return LBM_OK;
}

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

lbm_status lbm_mlp_create(int n_in, int width, int depth, int n_pos, int n_cls, int max_batch,
                          unsigned long long seed, void* cuda_stream, lbm_mlp** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (n_in < 1 || width < 1 || width > 4096 || depth < 1 || depth > 8 || n_pos < 0 || n_cls < 0 || n_cls > 64 ||
      n_pos + n_cls < 1 || max_batch < 1 || max_batch > (1 << 20))
    return LBM_EINVAL;
  lbm_mlp* m = new (std::nothrow) lbm_mlp();
  if (!m) return LBM_ENOMEM;
  m->n_in = n_in;
  m->width = width;
  m->depth = depth;
  m->n_pos = n_pos;
  m->n_cls = n_cls;
  m->n_out = n_pos + n_cls;
  m->max_batch = max_batch;
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  m->step = 0;
  const int L = depth + 1;
  size_t o = 0;
  for (int l = 0; l < L; ++l) {
    const int fi = l == 0 ? n_in : width, fo = l == L - 1 ? m->n_out : width;
    m->fan_in.push_back(fi);
    m->fan_out.push_back(fo);
    m->w_off.push_back(o);
    o += (size_t)fi * fo;
    m->b_off.push_back(o);
    o += (size_t)fo;
  }
  m->P = o;
  const size_t B = (size_t)max_batch, W = (size_t)width, wide = (size_t)(width > m->n_out ? width : m->n_out);
  size_t max_part = 0;
  for (int l = 0; l < L; ++l) {
    const size_t s = (size_t)((max_batch + KSPLIT - 1) / KSPLIT) * m->fan_in[l] * m->fan_out[l];
    if (s > max_part) max_part = s;
  }
  // one device allocation, carved into 256-byte aligned pieces
  std::vector<std::pair<void**, size_t>> parts;
  parts.push_back({(void**)&m->p, 4 * m->P});
  parts.push_back({(void**)&m->g, 4 * m->P});
  parts.push_back({(void**)&m->m, 4 * m->P});
  parts.push_back({(void**)&m->v, 4 * m->P});
  parts.push_back({(void**)&m->pb, 2 * m->P});
  parts.push_back({(void**)&m->x32, 4 * B * n_in});
  parts.push_back({(void**)&m->h[0], 2 * B * n_in});
  for (int l = 1; l <= depth; ++l) {
    parts.push_back({(void**)&m->h[l], 2 * B * W});
    parts.push_back({(void**)&m->z[l], 4 * B * W});
  }
  parts.push_back({(void**)&m->y, 4 * B * m->n_out});
  for (int k = 0; k < 2; ++k) {
    parts.push_back({(void**)&m->d32[k], 4 * B * wide});
    parts.push_back({(void**)&m->d16[k], 2 * B * wide});
  }
  parts.push_back({(void**)&m->part, 4 * max_part});
  parts.push_back({(void**)&m->tgt, 4 * B * (n_pos > 0 ? n_pos : 1)});
  parts.push_back({(void**)&m->row_loss, 4 * B});
  parts.push_back({(void**)&m->loss, 4});
  parts.push_back({(void**)&m->lab, 4 * B});
  parts.push_back({(void**)&m->bad, 4});
  size_t total = 0;
  for (auto& pr : parts) total += (pr.second + 255) / 256 * 256;
  if (cudaMalloc(&m->mem, total) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return LBM_ENOMEM;
  }
  size_t off = 0;
  for (auto& pr : parts) {
    *pr.first = m->mem + off;
    off += (pr.second + 255) / 256 * 256;
  }
  // parameters: uniform in +-1/sqrt(fan_in) (SplitMix64 stream from seed)
  std::vector<float> init(m->P);
  uint64_t s = seed;
  for (int l = 0; l < L; ++l) {
    const double a = 1.0 / sqrt((double)m->fan_in[l]);
    const size_t n = (size_t)m->fan_in[l] * m->fan_out[l] + m->fan_out[l];
    for (size_t i = 0; i < n; ++i)
      init[m->w_off[l] + i] = (float)(a * (2.0 * ((double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0)) - 1.0));
  }
  lbm_status st = lbm_mlp_set_params(m, init.data());
  if (st != LBM_OK) {
    lbm_mlp_free(m);
    return st;
  }
  *out = m;
  return LBM_OK;
}

size_t lbm_mlp_param_count(const lbm_mlp* m) { return m ? m->P : 0; }

lbm_status lbm_mlp_set_params(lbm_mlp* m, const float* params) {
  if (!m || !params) return LBM_EINVAL;
  const cudaMemcpyKind k = is_device_ptr(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  MLP_CUDA(cudaMemcpyAsync(m->p, params, 4 * m->P, k, m->stream));
  MLP_CUDA(cudaMemsetAsync(m->m, 0, 4 * m->P, m->stream));
  MLP_CUDA(cudaMemsetAsync(m->v, 0, 4 * m->P, m->stream));
  k_to_bf16<<<blocks((long long)m->P, 256), 256, 0, m->stream>>>(m->p, m->pb, (long long)m->P);
  MLP_CUDA(cudaGetLastError());
  m->step = 0;
  MLP_CUDA(cudaStreamSynchronize(m->stream));
  return LBM_OK;
}

lbm_status lbm_mlp_get_params(lbm_mlp* m, float* params) {
  if (!m || !params) return LBM_EINVAL;
  lbm_status st = copy_out(m, params, m->p, 4 * m->P);
  if (st != LBM_OK) return st;
  MLP_CUDA(cudaStreamSynchronize(m->stream));
  return LBM_OK;
}

lbm_status lbm_mlp_forward(lbm_mlp* m, const float* x, int batch, float* y) {
  if (!m || !x || !y || batch < 1 || batch > m->max_batch) return LBM_EINVAL;
  lbm_status st = stage_inputs(m, x, nullptr, nullptr, batch);
  if (st == LBM_OK) st = forward(m, batch);
  if (st == LBM_OK) st = copy_out(m, y, m->y, sizeof(float) * batch * m->n_out);
  if (st != LBM_OK) return st;
  MLP_CUDA(cudaStreamSynchronize(m->stream));
  return LBM_OK;
}

lbm_status lbm_mlp_loss_grad(lbm_mlp* m, const float* x, const float* target, const int* label, int batch,
                             float w_pos, float w_cls, float* loss, float* grad) {
  if (!m || !x || batch < 1 || batch > m->max_batch) return LBM_EINVAL;
  if ((m->n_pos > 0 && !target) || (m->n_cls > 0 && !label)) return LBM_EINVAL;
  lbm_status st = stage_inputs(m, x, target, label, batch);
  if (st == LBM_OK) st = backward(m, batch, w_pos, w_cls);
  if (st == LBM_OK && loss) st = copy_out(m, loss, m->loss, sizeof(float));
  if (st == LBM_OK && grad) st = copy_out(m, grad, m->g, 4 * m->P);
  if (st != LBM_OK) return st;
  int bad = 0;
  MLP_CUDA(cudaMemcpyAsync(&bad, m->bad, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  MLP_CUDA(cudaStreamSynchronize(m->stream));
  return bad ? LBM_EINVAL : LBM_OK;
}

lbm_status lbm_mlp_train_step(lbm_mlp* m, const float* x, const float* target, const int* label, int batch,
                              float w_pos, float w_cls, float lr, float* loss) {
  if (!m || !x || batch < 1 || batch > m->max_batch || !(lr >= 0.0f)) return LBM_EINVAL;
  if ((m->n_pos > 0 && !target) || (m->n_cls > 0 && !label)) return LBM_EINVAL;
  lbm_status st = stage_inputs(m, x, target, label, batch);
  if (st == LBM_OK) st = backward(m, batch, w_pos, w_cls);
  if (st != LBM_OK) return st;
  m->step += 1;
  const float c1 = (float)(1.0 - pow(0.9, (double)m->step)), c2 = (float)(1.0 - pow(0.999, (double)m->step));
  k_adam<<<blocks((long long)m->P, 256), 256, 0, m->stream>>>(m->p, m->g, m->m, m->v, m->pb, (long long)m->P, lr, c1,
                                                               c2);
  MLP_CUDA(cudaGetLastError());
  if (loss) {
    st = copy_out(m, loss, m->loss, sizeof(float));
    if (st != LBM_OK) return st;
  }
  int bad = 0;
  MLP_CUDA(cudaMemcpyAsync(&bad, m->bad, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  MLP_CUDA(cudaStreamSynchronize(m->stream));
  return bad ? LBM_EINVAL : LBM_OK;
}

void lbm_mlp_free(lbm_mlp* m) {
  if (!m) return;
  if (m->mem) cudaFree(m->mem);
  delete m;
}

}  // extern "C"
