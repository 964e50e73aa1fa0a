// Host implementation of the C ABI declared in include/lbm.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_dispatch.h"
#include "lbm_kernels.cuh"
#include "lbm_tma.cuh"

using lbmk::Geom;
using lbmk::KernelSet;
using lbmk::Phys;

namespace {

constexpr int kGraphSteps = 16;  // steps per captured CUDA graph

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {  // byte offsets inside the device workspace
  size_t pop, dens, fix, top, counter, flag, partial, diag_out, scratch, total;
};

}  // namespace

struct lbm {
  int nx, ny, nz;
  int64_t N;
  lbm_params p;
  const KernelSet* ks;
  Geom G;
  Phys P;
  Layout L;
  char* ws;
  bool own_ws;
  void *pop, *dens, *top, *partial;
  unsigned long long* fix[2];  // fused density pass: packed fixed-point (rho, rho_r) of the state at an even / odd step
  bool fix_ready;   // fix[t & 1] holds the densities of the current state
  long long* counter;  // [2]: step index, see k_collide_stream
  int* flag;
  double *diag_out, *scratch;
  int diag_blocks;
  int variant;  // pass-2 kernel: 1 = one node per thread, 2 = two nodes per thread, 3 = fused density
  int shape;    // block shape of the one-node kernels (lbm_params.block)
  cudaStream_t stream;
  cudaStream_t cap_stream;
  cudaGraphExec_t graph[2];  // kGraphSteps steps starting at an even / odd step
  long long graph_kernels[2];  // kernel launches one replay of graph[k] makes
  long long launches;          // kernel launches of this handle's steps so far (lbm_launch_count)
  long long t;
  bool unstable;
  bool timed_out;  // a bounded device-side wait ran out (flag bit kFlagTimeout)
  bool halo;     // a z face is LBM_BC_HALO: the handle is one slab of a decomposed domain
  bool recs_valid;  // compact storage: the colour records describe the current state
  bool dens_ready;  // compact storage: dens holds (rho, phi) of the current state
  int half;      // lbm_step_pass: 1 after pass 1 of the current step, 0 otherwise
  std::string err;
};

namespace {

lbm_status fail(lbm* h, lbm_status s, const char* fmt, ...) {
  if (h) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    h->err = buf;
  }
  return s;
}

#define LBM_CUDA(h, call)                                                                          \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail((h), LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

const KernelSet* kernels_for(int storage) {
  switch (storage) {
    case LBM_STORE_F64: return lbmk::kernels_f64();
    case LBM_STORE_F32: return lbmk::kernels_f32();
    case LBM_STORE_F16: return lbmk::kernels_f16();
    case LBM_STORE_BF16: return lbmk::kernels_bf16();
    case LBM_STORE_F16C: return lbmk::kernels_c16();
    case LBM_STORE_BF16C: return lbmk::kernels_cbf16();
    default: return nullptr;
  }
}

// where the pipelined compact pass 1 applies: x faces that reflect (free-slip), no row whose last
// 32-node block holds a single node (that lane would be both block edges), and at least three
// 32x4x2 tiles along y and z (the tiles next to the faces go to the one-block kernel)
bool pipelined_ok(int nx, int ny, int nz, const lbm_params* p) {
  return p->bc[0] != LBM_BC_PERIODIC && p->bc[1] != LBM_BC_PERIODIC && p->bc[0] != LBM_BC_NOSLIP &&
         p->bc[1] != LBM_BC_NOSLIP && nx % 32 != 1 && ny > 2 * lbmk::BY && nz > 2 * lbmk::BZ;
}

const char* validate(int nx, int ny, int nz, const lbm_params* p) {
  if (!p) return "params is NULL";
  if (nx < 3 || ny < 3 || nz < 3) return "each box dimension must be >= 3";
  if ((double)nx * ny * nz >= 2147483647.0 / 2) return "box too large (nx*ny*nz must stay below 2^30)";
  // the kernels address a node's slots by 32-bit offsets from its own: one z plane of storage
  // (up to 54 values per node) must hold fewer than 2^31 elements
  if ((double)align_up((size_t)nx, 32) * ny * 54.0 >= 2147483647.0 - 65536.0)
    return "xy plane too large (nx rounded up to 32, times ny, times 54 must stay below 2^31)";
  if (!(p->rho_r0 > 0) || !(p->rho_b0 > 0)) return "rho_r0 and rho_b0 must be > 0";
  const double ab = 8.0 / 27.0, ar = 1.0 - (1.0 - ab) / (p->rho_r0 / p->rho_b0);
  if (!(ar >= 0.0 && ar < 1.0)) return "density ratio rho_r0/rho_b0 must be >= 19/27 (alpha_r in [0,1))";
  if (!(p->nu_r > 0) || !(p->nu_b > 0)) return "nu_r and nu_b must be > 0";
  if (!(p->A >= 0) || !(p->beta >= 0 && p->beta <= 1)) return "need A >= 0 and 0 <= beta <= 1";
  for (int j = 4; j < 27; ++j) {
    if (j >= 5 && j <= 9) continue;  // shear slots come from the viscosity
    if (!(p->s[j] >= 0.0 && p->s[j] < 2.0)) return "relaxation rates must lie in [0, 2)";
    for (int k = 4; k < j; ++k)
      if (lbmk::kslot_of(k) == lbmk::kslot_of(j) && p->s[k] != p->s[j])
        return "moments of one relaxation slot of K must share one rate";
  }
  if (p->force_mode < 0 || p->force_mode > 3) return "unknown force_mode";
  for (int f = 0; f < 6; ++f)
    if (p->bc[f] < 0 || p->bc[f] > 5) return "unknown boundary code";
  for (int f = 0; f < 4; ++f)
    if (p->bc[f] == LBM_BC_HALO) return "HALO faces are only allowed on -z and +z";
  if ((p->bc[4] == LBM_BC_HALO || p->bc[5] == LBM_BC_HALO) && p->variant == 3)
    return "slab handles (HALO faces) do not run the fused density pass (variant 3)";
  for (int a = 0; a < 3; ++a)
    if ((p->bc[2 * a] == LBM_BC_PERIODIC) != (p->bc[2 * a + 1] == LBM_BC_PERIODIC))
      return "periodic faces must come in pairs";
  for (int f = 0; f < 6; ++f) {
    if (p->bc[f] == LBM_BC_INFLOW_WALL && f != 4) return "INFLOW_WALL is only allowed on the -z face";
    if (p->bc[f] == LBM_BC_OUTFLOW && f != 5) return "OUTFLOW is only allowed on the +z face";
  }
  if (p->storage < 0 || p->storage > 5) return "unknown storage";
  if (p->block < 0 || p->block > 4)
    return "unknown block shape (0: library's choice, 1: 32x4x2, 2: 32x2x4, 3: 32x8x1, 4: pipelined compact pass 1)";
  const bool compact = p->storage == LBM_STORE_F16C || p->storage == LBM_STORE_BF16C;
  if (compact) {
    if (p->variant > 1) return "compact storage runs the one-node collide-stream kernel (variant 0 or 1)";
    if (p->bc[4] == LBM_BC_HALO || p->bc[5] == LBM_BC_HALO) return "compact storage has no z-slab halo exchange";
    if (p->block == 2 || p->block == 3)
      return "compact storage runs 32x4x2 tiles: block 0, 1 or 4 (pipelined pass 1)";
  }
  if (p->block == 4 && !(compact && pipelined_ok(nx, ny, nz, p)))
    return "block 4 (TMA-pipelined pass 1) needs compact storage, x faces that are neither periodic nor no-slip, "
           "nx % 32 != 1, ny > 8 and nz > 4";
  if (p->variant < 0 || p->variant > 5) return "unknown kernel variant";
  if (p->variant == 4 && p->storage != LBM_STORE_F16 && p->storage != LBM_STORE_BF16)
    return "the software-pipelined kernel needs packed (F16/BF16) storage";
  if (p->variant == 5 && p->storage != LBM_STORE_F16 && p->storage != LBM_STORE_BF16)
    return "the TMA-pipelined kernel (variant 5) needs packed (F16/BF16) storage";
  if (p->variant == 2 && (p->storage == LBM_STORE_F64 || nx % 2 != 0))
    return "the two-nodes-per-thread kernel needs FP32 arithmetic (not F64 storage) and an even nx";
  if (p->variant == 3 && p->storage == LBM_STORE_F64)
    return "the fused density pass needs FP32 arithmetic (not F64 storage)";
  if (p->storage != LBM_STORE_F64 && (p->rho_r0 > 64.0 || p->rho_b0 > 64.0))
    return "FP32 storages need rho_r0, rho_b0 <= 64 (fixed-point range of the fused density pass)";
  return nullptr;
}

Layout plan(int nx, int ny, int nz, const lbm_params* p, const KernelSet* ks, int64_t* Ns_out, int* diag_blocks) {
  const int64_t N = (int64_t)nx * ny * nz;
  const int64_t nxs = (int64_t)align_up((size_t)nx, 32);  // storage rows: whole 32-node blocks
  const int64_t Ns = (int64_t)align_up((size_t)nxs * ny * (nz + 2), 64);
  const int64_t Pn = (int64_t)nx * ny;
  int nb = (int)((N + lbmk::DIAG_THREADS - 1) / lbmk::DIAG_THREADS);
  if (nb > 152 * 8) nb = 152 * 8;
  Layout L;
  size_t o = 0;
  L.pop = o;
  o = align_up(o + (size_t)Ns * ks->pop_node_bytes, 256);
  L.dens = o;  // (rho, phi) with one halo plane below and above (read only across HALO faces)
  o = align_up(o + (size_t)(N + 2 * Pn) * ks->dens_bytes, 256);
  L.fix = o;
  if (ks->has_fused) o = align_up(o + (size_t)4 * N * sizeof(int), 256);
  L.top = o;
  if (p->bc[5] == LBM_BC_OUTFLOW) o = align_up(o + (size_t)64 * Pn * ks->real_bytes, 256);
  L.counter = o;
  o = align_up(o + 2 * sizeof(long long), 256);
  L.flag = o;
  o = align_up(o + sizeof(int), 256);
  L.partial = o;
  o = align_up(o + (size_t)nb * lbmk::DIAG_VALS * sizeof(double), 256);
  L.diag_out = o;
  o = align_up(o + lbmk::DIAG_VALS * sizeof(double), 256);
  L.scratch = o;
  o = align_up(o + (size_t)5 * N * sizeof(double), 256);
  L.total = o;
  if (Ns_out) *Ns_out = Ns;
  if (diag_blocks) *diag_blocks = nb;
  return L;
}

__global__ void k_fill(double* a, int64_t n, double v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
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

void drop_graphs(lbm* h) {
  for (int k = 0; k < 2; ++k)
    if (h->graph[k]) {
      cudaGraphExecDestroy(h->graph[k]);
      h->graph[k] = nullptr;
    }
}

// variants with the fused density pass (no pass 1; fixed-point accumulators between steps)
bool fused_variant(const lbm* h) { return h->variant == 3; }

// enqueue one time step (the step with index t) on stream s; skip_density: the (rho, phi)
// field already holds the state's densities (first step of compact storage after an upload).
// Runs of two-pass steps with an outflow face (enqueue_run): fold, pass 1 first completes the
// step before with its convective outflow; last = false, the outflow kernel is left to the
// folding pass 1 of the next step.
lbm_status enqueue_step(lbm* h, long long t, cudaStream_t s, bool skip_density = false, bool fold = false,
                        bool last = true) {
  const int layout = (int)(t & 1);
  const bool outflow = h->p.bc[5] == LBM_BC_OUTFLOW;
  const long long ck = (h->variant == 5 && lbmk::pipelined_tiles(h->G)) ? 2 : 1;  // collide-stream launches
  if (fused_variant(h)) {
    // fused density pass: no pass 1; the accumulators of t+1 start from zero
    h->launches += ck + (outflow ? 1 : 0);
    unsigned long long *cur = h->fix[layout], *nxt = h->fix[layout ^ 1];
    LBM_CUDA(h, cudaMemsetAsync(nxt, 0, sizeof(unsigned long long) * (size_t)h->N, s));
    LBM_CUDA(h, h->ks->collide(h->pop, h->G, h->P, layout, h->dens, h->counter, h->variant, cur, nxt, h->flag,
                               h->shape, s));
    if (outflow) LBM_CUDA(h, h->ks->outflow(h->pop, h->G, h->P, layout ^ 1, h->top, nxt, s));
    return LBM_OK;
  }
  h->fix_ready = false;  // steps without the fused pass leave its accumulators behind
  h->launches += (skip_density ? 0 : 1) + ck + (outflow && last ? 1 : 0);
  if (!skip_density) {
    if (fold) LBM_CUDA(h, h->ks->density_fold(h->pop, h->G, h->P, layout, h->dens, h->flag, h->top, h->shape, s));
    else LBM_CUDA(h, h->ks->density(h->pop, h->G, h->P, layout, h->dens, h->flag, nullptr, h->shape, s));
  }
  LBM_CUDA(h, h->ks->collide(h->pop, h->G, h->P, layout, h->dens, h->counter, h->variant, nullptr, nullptr,
                             h->flag, h->shape, s));
  if (outflow && last) LBM_CUDA(h, h->ks->outflow(h->pop, h->G, h->P, layout ^ 1, h->top, nullptr, s));
  return LBM_OK;
}

// n >= 1 steps from step t0: with an outflow face, the two-pass schemes launch the outflow
// kernel only after the last step; each earlier step's outflow runs at the start of the next
// step's pass 1 (the same arithmetic), so the state after the run is the same
lbm_status enqueue_run(lbm* h, long long t0, int n, cudaStream_t s) {
  const bool fold = h->p.bc[5] == LBM_BC_OUTFLOW && !fused_variant(h) && h->ks->density_fold != nullptr;
  for (int k = 0; k < n; ++k) {
    lbm_status st = enqueue_step(h, t0 + k, s, false, fold && k > 0, !fold || k == n - 1);
    if (st != LBM_OK) return st;
  }
  return LBM_OK;
}

// before fused steps from a state the fused pass did not produce: fill the accumulators of step t
lbm_status ensure_fix(lbm* h, cudaStream_t s) {
  if (!fused_variant(h) || h->fix_ready) return LBM_OK;
  LBM_CUDA(h, h->ks->density(h->pop, h->G, h->P, (int)(h->t & 1), h->dens, h->flag, h->fix[h->t & 1], h->shape, s));
  h->fix_ready = true;
  return LBM_OK;
}

// the step index of step t for k_collide_stream
lbm_status set_counter(lbm* h, long long t) {
  LBM_CUDA(h, cudaMemcpyAsync(h->counter + (t & 1), &t, sizeof t, cudaMemcpyHostToDevice, h->stream));
  return LBM_OK;
}

lbm_status build_graph(lbm* h, int parity) {
  cudaGraph_t g = nullptr;
  LBM_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  lbm_status st = LBM_OK;
  const long long before = h->launches;  // captured, not launched: counted per replay
  st = enqueue_run(h, parity, kGraphSteps, h->cap_stream);
  h->graph_kernels[parity] = h->launches - before;
  h->launches = before;
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (st != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(h, LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->graph[parity], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->graph[parity] = nullptr;
    return fail(h, LBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  return LBM_OK;
}

// compact storage: the state uploaded by lbm_init_fields / lbm_set_populations has no colour
// records; its first step takes (rho, phi) as written by the upload instead of running pass 1
lbm_status compact_first_step(lbm* h, cudaStream_t s) {
  LBM_CUDA(h, cudaGetLastError());
  lbm_status st = enqueue_step(h, h->t, s, true);
  if (st != LBM_OK) return st;
  h->t += 1;
  h->recs_valid = true;
  h->dens_ready = false;
  return LBM_OK;
}

// compact storage: (rho, phi) of the current state in dens (pass 1, if not already there)
lbm_status compact_dens(lbm* h) {
  if (!h->ks->compact || h->dens_ready) return LBM_OK;
  LBM_CUDA(h, h->ks->density(h->pop, h->G, h->P, (int)(h->t & 1), h->dens, h->flag, nullptr, h->shape, h->stream));
  h->dens_ready = true;
  return LBM_OK;
}

// the errors a kernel reported through the flag stay with the handle until the next upload
lbm_status sticky_status(lbm* h) {
  if (h->timed_out) return fail(h, LBM_ETIMEOUT, "a bounded device-side wait of a pipelined kernel ran out");
  if (h->unstable) return fail(h, LBM_EUNSTABLE, "watchdog: non-finite or non-positive density seen");
  return LBM_OK;
}

lbm_status check_flag(lbm* h) {
  int flag = 0;
  LBM_CUDA(h, cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  if (flag & lbmk::kFlagTimeout) h->timed_out = true;
  if (flag & ~lbmk::kFlagTimeout) h->unstable = true;
  return sticky_status(h);
}

}  // namespace

extern "C" {

const char* lbm_status_string(lbm_status s) {
  switch (s) {
    case LBM_OK: return "LBM_OK";
    case LBM_EINVAL: return "LBM_EINVAL";
    case LBM_ENOMEM: return "LBM_ENOMEM";
    case LBM_ECUDA: return "LBM_ECUDA";
    case LBM_EUNSTABLE: return "LBM_EUNSTABLE";
    case LBM_ETIMEOUT: return "LBM_ETIMEOUT";
    case LBM_ESTATE: return "LBM_ESTATE";
  }
  return "unknown";
}

lbm_status lbm_workspace_size(int nx, int ny, int nz, const lbm_params* p, size_t* bytes) {
  if (!bytes || validate(nx, ny, nz, p)) return LBM_EINVAL;
  *bytes = plan(nx, ny, nz, p, kernels_for(p->storage), nullptr, nullptr).total;
  return LBM_OK;
}

lbm_status lbm_create(int nx, int ny, int nz, const lbm_params* p, lbm** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (validate(nx, ny, nz, p)) return LBM_EINVAL;
  lbm* h = new (std::nothrow) lbm();
  if (!h) return LBM_ENOMEM;
  h->nx = nx;
  h->ny = ny;
  h->nz = nz;
  h->N = (int64_t)nx * ny * nz;
  h->p = *p;
  h->ks = kernels_for(p->storage);
  int64_t Ns = 0;
  h->L = plan(nx, ny, nz, p, h->ks, &Ns, &h->diag_blocks);
  h->stream = static_cast<cudaStream_t>(p->cuda_stream);
  // default, as measured on GB300: FP32 storage runs the fused density pass when rows
  // fill whole 32-node blocks (its collide-stream kernel is bandwidth-bound, so dropping
  // the separate density pass pays; partial blocks would take the per-direction atomic
  // path); the packed storages run the two-pass scheme with the TMA-pipelined collide-stream
  // kernel on the interior tiles (variant 5: 0.384 against 0.394 ms for the one-node kernel on
  // the 128x128x512 jet; it runs variant 1 where it does not apply) and FP64 one node per
  // thread (the packed kernels are issue-bound, and the fused accumulation costs more
  // instructions than the density pass); the two-node kernel's register footprint
  // leaves 8 warps per SM and measured slower everywhere
  h->halo = p->bc[4] == LBM_BC_HALO || p->bc[5] == LBM_BC_HALO;
  h->half = 0;
  h->recs_valid = false;
  h->dens_ready = false;
  const bool packed = p->storage == LBM_STORE_F16 || p->storage == LBM_STORE_BF16;
  h->variant = p->variant != 0 ? p->variant
                               : (p->storage == LBM_STORE_F32 && nx % 32 == 0 && !h->halo ? 3 : (packed ? 5 : 1));
  h->fix_ready = false;
  // block shape: as measured on GB300 (128x128x512 jet), the fused FP32 kernel runs fastest in
  // 32x2x4 blocks (0.784 against 0.814 ms for 32x4x2); every other kernel in 32x4x2
  h->shape = p->block != 0 ? p->block - 1 : (h->variant == 3 && p->storage == LBM_STORE_F32 ? 1 : 0);
  // compact storage: the TMA-pipelined pass 1 wherever it applies (0.11 against 0.36 ms on the jet)
  if (h->ks->compact && p->block == 0 && pipelined_ok(nx, ny, nz, p)) h->shape = 3;

  Geom& G = h->G;
  G.nx = nx;
  G.nxs = (int)align_up((size_t)nx, 32);
  G.ny = ny;
  G.nz = nz;
  G.Ns = Ns;
  for (int f = 0; f < 6; ++f) G.bc[f] = p->bc[f];
  G.inflow = 0;
  G.xc = G.yc = G.r2 = 0.0;
  G.ctop = nullptr;

  Phys& P = h->P;
  memset(&P, 0, sizeof P);
  P.rho_r0 = p->rho_r0;
  P.rho_b0 = p->rho_b0;
  P.alpha_b = 8.0 / 27.0;  // Sec. II: alpha_b = 8/27, c_s^b = 1/sqrt(3)
  P.alpha_r = 1.0 - (1.0 - P.alpha_b) / (p->rho_r0 / p->rho_b0);  // gamma = (1-alpha_b)/(1-alpha_r)
  P.nu_r = p->nu_r;
  P.nu_b = p->nu_b;
  P.A = p->A;
  P.beta = p->beta;
  for (int j = 0; j < 27; ++j) P.rate[j] = (j < 4 || lbmk::is_shear_moment(j)) ? 0.0 : p->s[j];
  for (int a = 0; a < 3; ++a) P.g[a] = p->g[a];
  P.force_mode = p->force_mode;
  P.rho_ref = p->force_mode == LBM_FORCE_BUOYANCY ? 0.5 * (p->rho_r0 + p->rho_b0) : p->rho_b0;
  P.seed = p->seed;


  if (p->workspace) {
    if (p->workspace_bytes < h->L.total) {
      delete h;
      return LBM_ENOMEM;
    }
    if (((uintptr_t)p->workspace) % 256) {
      delete h;
      return LBM_EINVAL;
    }
    h->ws = static_cast<char*>(p->workspace);
    h->own_ws = false;
  } else {
    void* mem = nullptr;
    if (cudaMalloc(&mem, h->L.total) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return LBM_ENOMEM;
    }
    h->ws = static_cast<char*>(mem);
    h->own_ws = true;
  }
  h->pop = h->ws + h->L.pop;
  h->dens = h->ws + h->L.dens + (size_t)nx * ny * h->ks->dens_bytes;  // plane z = 0 (z = -1 below it)
  h->fix[0] = reinterpret_cast<unsigned long long*>(h->ws + h->L.fix);
  h->fix[1] = h->fix[0] + h->N;
  h->top = h->ws + h->L.top;
  if (h->ks->compact && p->bc[5] == LBM_BC_OUTFLOW) h->G.ctop = static_cast<float*>(h->top);
  h->counter = reinterpret_cast<long long*>(h->ws + h->L.counter);
  h->flag = reinterpret_cast<int*>(h->ws + h->L.flag);
  h->partial = h->ws + h->L.partial;
  h->diag_out = reinterpret_cast<double*>(h->ws + h->L.diag_out);
  h->scratch = reinterpret_cast<double*>(h->ws + h->L.scratch);
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    if (h->own_ws) cudaFree(h->ws);
    delete h;
    return LBM_ECUDA;
  }
  if (h->ks->compact &&  // colour records: defined contents before the first step writes them
      cudaMemsetAsync(static_cast<char*>(h->pop) + (size_t)56 * h->G.Ns, 0, (size_t)16 * h->G.Ns, h->stream) !=
          cudaSuccess) {
    cudaGetLastError();
    lbm_free(h);
    return LBM_ECUDA;
  }
  // initial state: pure blue fluid at rest
  {
    double* rr = h->scratch;
    double* rb = h->scratch + h->N;
    const unsigned nb = (unsigned)((h->N + 255) / 256);
    k_fill<<<nb, 256, 0, h->stream>>>(rr, h->N, 0.0);
    k_fill<<<nb, 256, 0, h->stream>>>(rb, h->N, p->rho_b0);
    lbm_status st = cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
    if (st == LBM_OK) st = lbm_init_fields(h, rr, rb, nullptr);
    if (st != LBM_OK) {
      cudaGetLastError();
      lbm_free(h);
      return st;
    }
  }
  *out = h;
  return LBM_OK;
}

lbm_status lbm_init_fields(lbm* h, const double* rhoR, const double* rhoB, const double* u) {
  if (!h) return LBM_EINVAL;
  if (!rhoR || !rhoB) return fail(h, LBM_EINVAL, "rhoR and rhoB are required");
  const int64_t N = h->N;
  const double *dr = rhoR, *db = rhoB, *du = u;
  double* sr = h->scratch;
  double* sb = h->scratch + N;
  double* su = h->scratch + 2 * N;
  // stage host inputs (device inputs may alias the scratch: copy them in order)
  if (!is_device_ptr(rhoR)) {
    LBM_CUDA(h, cudaMemcpyAsync(sr, rhoR, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
    dr = sr;
  }
  if (!is_device_ptr(rhoB)) {
    LBM_CUDA(h, cudaMemcpyAsync(sb, rhoB, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
    db = sb;
  }
  if (u && !is_device_ptr(u)) {
    LBM_CUDA(h, cudaMemcpyAsync(su, u, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, h->stream));
    du = su;
  }
  if (h->ks->compact) {
    // totals, (rho, phi) and the top plane's colours; the first step takes (rho, phi) as given
    LBM_CUDA(h, h->ks->init_c(h->pop, h->G, h->P, dr, db, du, h->dens, h->stream));
    h->dens_ready = true;
    h->recs_valid = false;
  } else {
    LBM_CUDA(h, h->ks->init(h->pop, h->G, h->P, dr, db, du, h->stream));
  }
  h->t = 0;
  h->half = 0;
  h->fix_ready = false;
  {
    lbm_status st = set_counter(h, 0);
    if (st != LBM_OK) return st;
  }
  LBM_CUDA(h, cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
  if (h->p.bc[5] == LBM_BC_OUTFLOW && !h->ks->compact)
    LBM_CUDA(h, h->ks->top_from_state(h->pop, h->G, h->P, 0, h->top, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->unstable = false;
  h->timed_out = false;
  return LBM_OK;
}

lbm_status lbm_set_inflow(lbm* h, double xc, double yc, double D, double u_j0, double noise_frac) {
  if (!h) return LBM_EINVAL;
  if (h->p.bc[4] != LBM_BC_INFLOW_WALL) return fail(h, LBM_ESTATE, "the -z face is not LBM_BC_INFLOW_WALL");
  if (!(isfinite(xc) && isfinite(yc) && isfinite(D) && isfinite(u_j0) && isfinite(noise_frac)) || noise_frac < 0)
    return fail(h, LBM_EINVAL, "inlet parameters must be finite, noise_frac >= 0");
  if (!(fabs(u_j0) < 0.5)) return fail(h, LBM_EINVAL, "|u_j0| must stay below 0.5 lattice units");
  h->G.inflow = D > 0 ? 1 : 0;
  h->G.xc = xc;
  h->G.yc = yc;
  h->G.r2 = D > 0 ? 0.25 * D * D : 0.0;
  h->P.u_j0 = u_j0;
  h->P.noise_frac = noise_frac;
  drop_graphs(h);
  return LBM_OK;
}

lbm_status lbm_step(lbm* h, int n) {
  if (!h || n < 0) return h ? fail(h, LBM_EINVAL, "n must be >= 0") : LBM_EINVAL;
  if (h->unstable || h->timed_out) return sticky_status(h);
  if (h->halo) return fail(h, LBM_ESTATE, "slab handles (HALO faces) step with lbm_step_pass and halo exchanges");
  if (h->half) return fail(h, LBM_ESTATE, "a step begun with lbm_step_pass(h, 1) must end with lbm_step_pass(h, 2)");
  static const bool no_graphs = getenv("LBM_NO_GRAPHS") != nullptr;
  {
    lbm_status st = ensure_fix(h, h->stream);
    if (st != LBM_OK) return st;
  }
  int k = 0;
  if (h->ks->compact && n > 0) {
    if (!h->recs_valid) {
      lbm_status st = compact_first_step(h, h->stream);
      if (st != LBM_OK) return st;
      k = 1;
    }
    h->dens_ready = false;
  }
  if (!no_graphs && n >= kGraphSteps) {
    const int parity = (int)(h->t & 1);
    if (!h->graph[parity]) {
      lbm_status st = build_graph(h, parity);
      if (st != LBM_OK) return st;
    }
    for (; k + kGraphSteps <= n; k += kGraphSteps) {
      LBM_CUDA(h, cudaGraphLaunch(h->graph[parity], h->stream));
      h->t += kGraphSteps;
      h->launches += h->graph_kernels[parity];
    }
  }
  if (k < n) {
    lbm_status st = enqueue_run(h, h->t, n - k, h->stream);
    if (st != LBM_OK) return st;
    h->t += n - k;
  }
  return LBM_OK;
}

lbm_status lbm_macro(lbm* h, double* rhoR, double* rhoB, double* u) {
  if (!h) return LBM_EINVAL;
  const int64_t N = h->N;
  const int layout = (int)(h->t & 1);
  double* dr = rhoR ? (is_device_ptr(rhoR) ? rhoR : h->scratch) : nullptr;
  double* db = rhoB ? (is_device_ptr(rhoB) ? rhoB : h->scratch + N) : nullptr;
  double* du = u ? (is_device_ptr(u) ? u : h->scratch + 2 * N) : nullptr;
  if (h->ks->compact) {
    lbm_status st = compact_dens(h);
    if (st != LBM_OK) return st;
    LBM_CUDA(h, h->ks->macro_c(h->pop, h->G, h->P, layout, h->dens, dr, db, du, h->stream));
  } else {
    LBM_CUDA(h, h->ks->macro(h->pop, h->G, h->P, layout, dr, db, du, h->stream));
  }
  if (rhoR && dr != rhoR) LBM_CUDA(h, cudaMemcpyAsync(rhoR, dr, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream));
  if (rhoB && db != rhoB) LBM_CUDA(h, cudaMemcpyAsync(rhoB, db, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream));
  if (u && du != u) LBM_CUDA(h, cudaMemcpyAsync(u, du, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, h->stream));
  return check_flag(h);
}

lbm_status lbm_diag(lbm* h, double* mass_rb, double* z_leading_edge, double* dp_laplace) {
  if (!h) return LBM_EINVAL;
  const int64_t N = h->N;
  const int layout = (int)(h->t & 1);
  double* rr = h->scratch;
  double* rb = h->scratch + N;
  if (h->ks->compact) {
    lbm_status st = compact_dens(h);
    if (st != LBM_OK) return st;
    LBM_CUDA(h, h->ks->macro_c(h->pop, h->G, h->P, layout, h->dens, rr, rb, nullptr, h->stream));
  } else {
    LBM_CUDA(h, h->ks->macro(h->pop, h->G, h->P, layout, rr, rb, nullptr, h->stream));
  }
  lbmk::k_diag_partial<<<h->diag_blocks, lbmk::DIAG_THREADS, 0, h->stream>>>(
      h->G, h->P.alpha_r, h->P.alpha_b, rr, rb, static_cast<double*>(h->partial));
  LBM_CUDA(h, cudaGetLastError());
  lbmk::k_diag_final<<<1, 32 * lbmk::DIAG_VALS, 0, h->stream>>>(h->diag_blocks, static_cast<double*>(h->partial),
                                                                 h->diag_out);
  LBM_CUDA(h, cudaGetLastError());
  double v[lbmk::DIAG_VALS];
  LBM_CUDA(h, cudaMemcpyAsync(v, h->diag_out, sizeof v, cudaMemcpyDeviceToHost, h->stream));
  lbm_status st = check_flag(h);
  if (st != LBM_OK) return st;
  if (mass_rb) {
    mass_rb[0] = v[0];
    mass_rb[1] = v[1];
  }
  if (z_leading_edge) *z_leading_edge = v[6];
  if (dp_laplace) *dp_laplace = (v[3] > 0 && v[5] > 0) ? v[2] / v[3] - v[4] / v[5] : 0.0;
  return LBM_OK;
}

lbm_status lbm_get_populations(lbm* h, double* f) {
  if (!h) return LBM_EINVAL;
  if (!f) return fail(h, LBM_EINVAL, "f is NULL");
  if (h->ks->compact && !h->recs_valid)
    return fail(h, LBM_ESTATE, "compact storage holds the colours of an uploaded state only after its first step");
  const int64_t N = h->N;
  const int layout = (int)(h->t & 1);
  const bool dev = is_device_ptr(f);
  for (int i = 0; i < 27; ++i) {
    double* outr = dev ? f + (int64_t)i * N : h->scratch;
    double* outb = dev ? f + (int64_t)(27 + i) * N : h->scratch + N;
    LBM_CUDA(h, h->ks->get_pop(h->pop, h->G, h->P, layout, i, outr, outb, h->stream));
    if (!dev) {
      LBM_CUDA(h, cudaMemcpyAsync(f + (int64_t)i * N, outr, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream));
      LBM_CUDA(h, cudaMemcpyAsync(f + (int64_t)(27 + i) * N, outb, sizeof(double) * N, cudaMemcpyDeviceToHost,
                                  h->stream));
    }
  }
  return check_flag(h);
}

lbm_status lbm_set_populations(lbm* h, const double* f, long long t) {
  if (!h) return LBM_EINVAL;
  if (!f || t < 0) return fail(h, LBM_EINVAL, "f is NULL or t < 0");
  const int64_t N = h->N;
  const int layout = (int)(t & 1);
  const bool dev = is_device_ptr(f);
  for (int i = 0; i < 27; ++i) {
    const double* inr = f + (int64_t)i * N;
    const double* inb = f + (int64_t)(27 + i) * N;
    if (!dev) {
      LBM_CUDA(h, cudaMemcpyAsync(h->scratch, inr, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
      LBM_CUDA(h, cudaMemcpyAsync(h->scratch + N, inb, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
      inr = h->scratch;
      inb = h->scratch + N;
    }
    if (h->ks->compact)
      LBM_CUDA(h, h->ks->set_pop_c(h->pop, h->G, h->P, layout, i, inr, inb, h->scratch + 2 * N, h->scratch + 3 * N,
                                   h->stream));
    else
      LBM_CUDA(h, h->ks->set_pop(h->pop, h->G, h->P, layout, i, inr, inb, h->stream));
  }
  if (h->ks->compact) {
    LBM_CUDA(h, h->ks->dens_from_acc(h->G, h->scratch + 2 * N, h->scratch + 3 * N, h->dens, h->stream));
    h->dens_ready = true;
    h->recs_valid = false;
  }
  h->t = t;
  h->half = 0;
  h->fix_ready = false;
  {
    lbm_status st = set_counter(h, t);
    if (st != LBM_OK) return st;
  }
  LBM_CUDA(h, cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
  if (h->p.bc[5] == LBM_BC_OUTFLOW && !h->ks->compact)
    LBM_CUDA(h, h->ks->top_from_state(h->pop, h->G, h->P, layout, h->top, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->unstable = false;
  h->timed_out = false;
  return LBM_OK;
}

lbm_status lbm_profile_step(lbm* h, int n, double* ms_out) {
  if (!h) return LBM_EINVAL;
  if (n < 1 || !ms_out) return fail(h, LBM_EINVAL, "need n >= 1 and an output array of 3 doubles");
  if (h->unstable || h->timed_out) return sticky_status(h);
  if (h->halo || h->half) return fail(h, LBM_ESTATE, "not available on slab handles or between step passes");
  if (h->ks->compact && !h->recs_valid)
    return fail(h, LBM_ESTATE, "compact storage: take one lbm_step after an upload before profiling");
  if (h->ks->compact) h->dens_ready = false;
  const bool outflow = h->p.bc[5] == LBM_BC_OUTFLOW;
  const int per = 4;
  cudaEvent_t* ev = (cudaEvent_t*)calloc((size_t)per * n, sizeof(cudaEvent_t));
  if (!ev) return fail(h, LBM_ENOMEM, "event array");
  lbm_status st = LBM_OK;
  int made = 0;
  for (; made < per * n; ++made)
    if (cudaEventCreate(&ev[made]) != cudaSuccess) {
      st = fail(h, LBM_ECUDA, "cudaEventCreate failed");
      break;
    }
  if (st == LBM_OK) st = ensure_fix(h, h->stream);
  const bool fused = fused_variant(h);
  if (!fused) h->fix_ready = false;
  for (int k = 0; st == LBM_OK && k < n; ++k) {
    const long long t = h->t;
    const int layout = (int)(t & 1);
    cudaEvent_t* e = ev + per * k;
    // the same launches as enqueue_step, with an event between them; with the fused density
    // pass the first interval is the clearing of the next step's accumulators
    unsigned long long* cur = h->fix[layout];
    unsigned long long* nxt = h->fix[layout ^ 1];
    const size_t nfix = sizeof(unsigned long long) * (size_t)h->N;
    if (cudaEventRecord(e[0], h->stream) != cudaSuccess ||
        (fused ? cudaMemsetAsync(nxt, 0, nfix, h->stream)
               : h->ks->density(h->pop, h->G, h->P, layout, h->dens, h->flag, nullptr, h->shape, h->stream)) !=
            cudaSuccess ||
        cudaEventRecord(e[1], h->stream) != cudaSuccess ||
        h->ks->collide(h->pop, h->G, h->P, layout, h->dens, h->counter, h->variant, fused ? cur : nullptr,
                       fused ? nxt : nullptr, h->flag, h->shape, h->stream) != cudaSuccess ||
        cudaEventRecord(e[2], h->stream) != cudaSuccess ||
        (outflow && h->ks->outflow(h->pop, h->G, h->P, layout ^ 1, h->top, fused ? nxt : nullptr, h->stream) !=
                        cudaSuccess) ||
        cudaEventRecord(e[3], h->stream) != cudaSuccess) {
      st = fail(h, LBM_ECUDA, "profiled step launch: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    h->t += 1;
  }
  if (st == LBM_OK && cudaStreamSynchronize(h->stream) != cudaSuccess)
    st = fail(h, LBM_ECUDA, "synchronize: %s", cudaGetErrorString(cudaGetLastError()));
  if (st == LBM_OK) {
    double acc[3] = {0, 0, 0};
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < 3; ++j) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[per * k + j], ev[per * k + j + 1]);
        acc[j] += ms;
      }
    for (int j = 0; j < 3; ++j) ms_out[j] = acc[j] / n;
    if (!outflow) ms_out[2] = 0.0;
  }
  for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
  free(ev);
  if (st != LBM_OK) return st;
  return check_flag(h);
}

lbm_status lbm_set_stream(lbm* h, void* cuda_stream) {
  if (!h) return LBM_EINVAL;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->p.cuda_stream = cuda_stream;
  return LBM_OK;
}

lbm_status lbm_synchronize(lbm* h) {
  if (!h) return LBM_EINVAL;
  return check_flag(h);
}

long long lbm_time(const lbm* h) { return h ? h->t : -1; }

int lbm_kernels_per_step(const lbm* h) {
  if (!h) return -1;
  // variant 5 launches two collide-stream kernels (boundary and interior tiles) where it applies
  const bool two = h->variant == 5 && lbmk::pipelined_tiles(h->G);
  return (fused_variant(h) ? 1 : 2) + (two ? 1 : 0) + (h->p.bc[5] == LBM_BC_OUTFLOW ? 1 : 0);
}

int lbm_kernel_variant(const lbm* h) { return h ? h->variant : -1; }

long long lbm_launch_count(const lbm* h) { return h ? h->launches : -1; }

int lbm_kernel_block(const lbm* h) { return h ? h->shape + 1 : -1; }

const char* lbm_last_error(const lbm* h) { return h ? h->err.c_str() : "NULL handle"; }

lbm_status lbm_moment_matrix(double* M) {
  if (!M) return LBM_EINVAL;
  static double Mt[27][27];
  lbmk::moment_matrix_tensor(Mt);
  for (int j = 0; j < 27; ++j)
    for (int i = 0; i < 27; ++i) M[27 * j + i] = Mt[j][lbmk::paper_to_tensor(i)];
  return LBM_OK;
}

lbm_status lbm_selfcheck(const char** msg) {
  static char buf[256];
  const char* ok = "ok";
  if (msg) *msg = ok;
  static double M[27][27];
  lbmk::moment_matrix_tensor(M);
  // every paper direction maps to a distinct tensor index
  int seen[27] = {0};
  for (int i = 0; i < 27; ++i) seen[lbmk::paper_to_tensor(i)]++;
  for (int t = 0; t < 27; ++t)
    if (seen[t] != 1) {
      if (msg) *msg = "paper_to_tensor is not a permutation";
      return LBM_EINVAL;
    }
  // rows 1-4 are the conserved moments <1>, <c_x>, <c_y>, <c_z>
  for (int t = 0; t < 27; ++t) {
    const double want[4] = {1.0, (double)lbmk::cx_of(t), (double)lbmk::cy_of(t), (double)lbmk::cz_of(t)};
    for (int j = 0; j < 4; ++j)
      if (M[j][t] != want[j]) {
        snprintf(buf, sizeof buf, "row %d of M is not the conserved moment", j + 1);
        if (msg) *msg = buf;
        return LBM_EINVAL;
      }
  }
  // rows mutually orthogonal (the inverse used by the kernels relies on it)
  for (int a = 0; a < 27; ++a)
    for (int b = 0; b < a; ++b) {
      double s = 0.0;
      for (int t = 0; t < 27; ++t) s += M[a][t] * M[b][t];
      if (s != 0.0) {
        snprintf(buf, sizeof buf, "rows %d and %d of M are not orthogonal", a + 1, b + 1);
        if (msg) *msg = buf;
        return LBM_EINVAL;
      }
    }
  // weights: sum 1, second moment 1/3
  double sw = 0.0, s2 = 0.0;
  for (int t = 0; t < 27; ++t) {
    sw += lbmk::weight_of(t);
    s2 += lbmk::weight_of(t) * lbmk::cx_of(t) * lbmk::cx_of(t);
  }
  if (fabs(sw - 1.0) > 1e-15 || fabs(s2 - 1.0 / 3.0) > 1e-15) {
    if (msg) *msg = "weights do not satisfy sum w = 1, sum w c_x^2 = 1/3";
    return LBM_EINVAL;
  }
  return LBM_OK;
}

lbm_status lbm_autotune(lbm* h, int steps, int* chosen) {
  if (!h) return LBM_EINVAL;
  if (steps < 1) return fail(h, LBM_EINVAL, "steps must be >= 1");
  if (h->unstable || h->timed_out) return sticky_status(h);
  if (h->halo || h->half) return fail(h, LBM_ESTATE, "not available on slab handles or between step passes");
  if (h->ks->compact && !h->recs_valid)
    return fail(h, LBM_ESTATE, "compact storage: take one lbm_step after an upload before autotuning");
  if (h->ks->compact) h->dens_ready = false;
  // candidates: (variant, block shape); the shapes apply to the one-node kernels (variants 1, 3)
  // of the FP32-arithmetic storages; compact storage: one-block or pipelined pass 1
  int cand[12][2], nc = 0;
  const bool shapes = !h->ks->compact && h->p.storage != LBM_STORE_F64;
  for (int v = 1; v <= 5; ++v) {
    if (v == 2 && !(h->ks->has_paired && h->nx % 2 == 0 && !h->ks->compact)) continue;
    if (v == 3 && !h->ks->has_fused) continue;
    if ((v == 4 || v == 5) && !h->ks->has_pipelined) continue;
    for (int b = 0; b < ((v == 1 || v == 3) && shapes ? 3 : 1); ++b) {
      cand[nc][0] = v;
      cand[nc][1] = b;
      ++nc;
    }
  }
  if (h->ks->compact && pipelined_ok(h->nx, h->ny, h->nz, &h->p)) {
    cand[nc][0] = 1;
    cand[nc][1] = 3;
    ++nc;
  }
  float ms[12] = {0.f};
  cudaEvent_t e0, e1;
  LBM_CUDA(h, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(h, LBM_ECUDA, "cudaEventCreate failed");
  }
  lbm_status st = LBM_OK;
  for (int c = 0; c < nc && st == LBM_OK; ++c) {
    if (h->variant != cand[c][0]) h->fix_ready = false;
    h->variant = cand[c][0];
    h->shape = cand[c][1];
    st = ensure_fix(h, h->stream);  // untimed: only needed when entering the fused pass
    // direct launches: every kernel timed the same way, no graph capture in between
    if (st == LBM_OK && cudaEventRecord(e0, h->stream) != cudaSuccess)
      st = fail(h, LBM_ECUDA, "cudaEventRecord failed");
    st = enqueue_run(h, h->t, steps, h->stream);
    if (st == LBM_OK) h->t += steps;
    if (st == LBM_OK && (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms[c], e0, e1) != cudaSuccess))
      st = fail(h, LBM_ECUDA, "autotune timing: %s", cudaGetErrorString(cudaGetLastError()));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LBM_OK) return st;
  int best = 0;
  for (int c = 1; c < nc; ++c)
    if (ms[c] < ms[best]) best = c;
  if (h->variant != cand[best][0]) h->fix_ready = false;
  h->variant = cand[best][0];
  h->shape = cand[best][1];
  drop_graphs(h);  // captured graphs hold the kernel of the previous choice
  if (chosen) *chosen = h->variant;
  return check_flag(h);
}

lbm_status lbm_step_pass(lbm* h, int pass) {
  if (!h) return LBM_EINVAL;
  if (pass != 1 && pass != 2) return fail(h, LBM_EINVAL, "pass must be 1 or 2");
  if (h->unstable || h->timed_out) return sticky_status(h);
  if (pass != h->half + 1) return fail(h, LBM_ESTATE, "passes must alternate 1, 2, 1, 2, ...");
  const long long t = h->t;
  const int layout = (int)(t & 1);
  cudaStream_t s = h->stream;
  if (pass == 1) {
    if (h->ks->compact && !h->recs_valid) {  // an uploaded state: (rho, phi) is already in dens
      h->half = 1;
      return LBM_OK;
    }
    if (fused_variant(h)) {
      lbm_status st = ensure_fix(h, s);
      if (st != LBM_OK) return st;
      LBM_CUDA(h, cudaMemsetAsync(h->fix[layout ^ 1], 0, sizeof(unsigned long long) * (size_t)h->N, s));
    } else {
      h->fix_ready = false;
      LBM_CUDA(h, h->ks->density(h->pop, h->G, h->P, layout, h->dens, h->flag, nullptr, h->shape, s));
    }
    h->half = 1;
    return LBM_OK;
  }
  const bool fused = fused_variant(h);
  LBM_CUDA(h, h->ks->collide(h->pop, h->G, h->P, layout, h->dens, h->counter, h->variant,
                             fused ? h->fix[layout] : nullptr, fused ? h->fix[layout ^ 1] : nullptr, h->flag, h->shape,
                             s));
  if (h->p.bc[5] == LBM_BC_OUTFLOW)
    LBM_CUDA(h, h->ks->outflow(h->pop, h->G, h->P, layout ^ 1, h->top, fused ? h->fix[layout ^ 1] : nullptr, s));
  h->t += 1;
  h->half = 0;
  h->recs_valid = true;
  h->dens_ready = false;
  return LBM_OK;
}

lbm_status lbm_halo_bytes(const lbm* h, int phase, size_t* bytes) {
  if (!h || !bytes) return LBM_EINVAL;
  const size_t plane = (size_t)h->nx * h->ny;
  if (phase == LBM_HALO_DENS) {
    *bytes = plane * h->ks->dens_bytes;
    return LBM_OK;
  }
  if (phase == LBM_HALO_POP_IN || phase == LBM_HALO_POP_OUT) {
    // 9 directions per stored colour plane set, whole 32-node storage blocks of one z plane
    *bytes = (size_t)h->ks->pop_planes * 9 * (size_t)h->G.nxs * h->ny * h->ks->pop_elem_bytes;
    return LBM_OK;
  }
  return LBM_EINVAL;
}

namespace {

// One face's message: the slots of one z plane that hold the populations moving across the
// face from the packing slab to the unpacking one (down through the packer's -z face, up
// through its +z face), 9 directions per stored colour.
//   POP_IN  (after an even step, layout 1: a slot's stored direction is opposite to the motion
//           of the population it holds) pack: the boundary plane; unpack: the ghost plane.
//   POP_OUT (after an odd step, layout 0: stored direction = motion) pack: the ghost plane the
//           odd step wrote into; unpack: the boundary plane.
// Stored directions are in tensor order t = (cx+1) + 3(cy+1) + 9(cz+1): c_z = -1 is t = 0..8,
// c_z = +1 is t = 18..26.
lbm_status halo_copy(lbm* h, int face, int phase, bool pack, char* buf) {
  if (face != 4 && face != 5) return fail(h, LBM_EINVAL, "face must be 4 (-z) or 5 (+z)");
  if (h->p.bc[face] != LBM_BC_HALO) return fail(h, LBM_ESTATE, "face %d is not LBM_BC_HALO", face);
  if (!buf) return fail(h, LBM_EINVAL, "buffer is NULL");
  cudaStream_t s = h->stream;
  const bool lo = face == 4;
  if (phase == LBM_HALO_DENS) {
    const size_t plane = (size_t)h->nx * h->ny * h->ks->dens_bytes;
    // pack: the plane next to the face; unpack: the halo plane beyond it
    const long long z = pack ? (lo ? 0 : h->nz - 1) : (lo ? -1 : h->nz);
    char* d = static_cast<char*>(h->dens) + z * (long long)plane;
    if (pack) LBM_CUDA(h, cudaMemcpyAsync(buf, d, plane, cudaMemcpyDeviceToDevice, s));
    else LBM_CUDA(h, cudaMemcpyAsync(d, buf, plane, cudaMemcpyDeviceToDevice, s));
    return LBM_OK;
  }
  if (phase != LBM_HALO_POP_IN && phase != LBM_HALO_POP_OUT) return fail(h, LBM_EINVAL, "unknown halo phase");
  const bool in = phase == LBM_HALO_POP_IN;
  const bool boundary = in == pack;  // the boundary plane (else the ghost plane beyond the face)
  const int z = boundary ? (lo ? 0 : h->nz - 1) : (lo ? -1 : h->nz);
  const bool down = pack ? lo : !lo;  // the message's populations move towards -z
  const bool stored_down = in ? !down : down;
  const int t0 = stored_down ? 0 : 18;
  const size_t e = h->ks->pop_elem_bytes;
  const int planes = 27 * h->ks->pop_planes;
  const size_t nblocks = (size_t)h->G.nxs * h->ny / 32;
  const size_t block0 = (size_t)h->G.nxs * h->ny * (size_t)(z + 1) / 32;  // storage plane z + 1
  const size_t width = 9 * 32 * e, spitch = (size_t)planes * 32 * e;
  for (int c = 0; c < h->ks->pop_planes; ++c) {
    char* slab = static_cast<char*>(h->pop) + (block0 * planes + (size_t)(c * 27 + t0)) * 32 * e;
    char* msg = buf + (size_t)c * nblocks * width;
    if (pack)
      LBM_CUDA(h, cudaMemcpy2DAsync(msg, width, slab, spitch, width, nblocks, cudaMemcpyDeviceToDevice, s));
    else
      LBM_CUDA(h, cudaMemcpy2DAsync(slab, spitch, msg, width, width, nblocks, cudaMemcpyDeviceToDevice, s));
  }
  return LBM_OK;
}

}  // namespace

lbm_status lbm_halo_pack(lbm* h, int face, int phase, void* buf) {
  if (!h) return LBM_EINVAL;
  return halo_copy(h, face, phase, true, static_cast<char*>(buf));
}

lbm_status lbm_halo_unpack(lbm* h, int face, int phase, const void* buf) {
  if (!h) return LBM_EINVAL;
  return halo_copy(h, face, phase, false, const_cast<char*>(static_cast<const char*>(buf)));
}

void lbm_free(lbm* h) {
  if (!h) return;
  drop_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->own_ws && h->ws) cudaFree(h->ws);
  delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batches: one graph with an independent branch per handle

struct lbm_batch {
  std::vector<lbm*> h;
  cudaStream_t stream;
  cudaStream_t root;                 // capture root
  std::vector<cudaStream_t> branch;  // one capture stream per handle
  cudaGraphExec_t graph[2];          // kGraphSteps steps from an even / odd parity
  std::vector<cudaEvent_t> ready;    // per handle: its own stream's work so far
  cudaEvent_t done;                  // the batch stream's work so far
  std::string err;
};

namespace {

void batch_drop(lbm_batch* b) {
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) {
      cudaGraphExecDestroy(b->graph[k]);
      b->graph[k] = nullptr;
    }
}

lbm_status batch_build(lbm_batch* b, int parity) {
  cudaGraph_t g = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins(b->h.size(), nullptr);
  lbm_status st = LBM_OK;
  if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) return LBM_ECUDA;
  for (auto& e : joins)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) st = LBM_ECUDA;
  if (st == LBM_OK && cudaStreamBeginCapture(b->root, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = LBM_ECUDA;
  if (st == LBM_OK) {
    cudaEventRecord(fork, b->root);
    for (size_t i = 0; i < b->h.size() && st == LBM_OK; ++i) {
      cudaStreamWaitEvent(b->branch[i], fork, 0);
      if (st == LBM_OK) {
        const long long before = b->h[i]->launches;  // captured: counted per replay
        st = enqueue_run(b->h[i], parity, kGraphSteps, b->branch[i]);
        b->h[i]->graph_kernels[parity] = b->h[i]->launches - before;
        b->h[i]->launches = before;
      }
      cudaEventRecord(joins[i], b->branch[i]);
      cudaStreamWaitEvent(b->root, joins[i], 0);
    }
    cudaError_t e = cudaStreamEndCapture(b->root, &g);
    if (st == LBM_OK && e != cudaSuccess) st = LBM_ECUDA;
  }
  if (st == LBM_OK && cudaGraphInstantiate(&b->graph[parity], g, 0) != cudaSuccess) {
    b->graph[parity] = nullptr;
    st = LBM_ECUDA;
  }
  if (g) cudaGraphDestroy(g);
  cudaEventDestroy(fork);
  for (auto& e : joins)
    if (e) cudaEventDestroy(e);
  if (st != LBM_OK) {
    cudaGetLastError();
    b->err = "batch graph capture failed";
  }
  return st;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(lbm* const* handles, int n, void* cuda_stream, lbm_batch** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!handles || n < 1) return LBM_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!handles[i] || handles[i]->halo) return LBM_EINVAL;
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ENOMEM;
  b->h.assign(handles, handles + n);
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->graph[0] = b->graph[1] = nullptr;
  b->root = nullptr;
  bool ok = cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking) == cudaSuccess;
  b->done = nullptr;
  b->branch.assign(n, nullptr);
  b->ready.assign(n, nullptr);
  for (int i = 0; i < n && ok; ++i) ok = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; i < n && ok; ++i) ok = cudaEventCreateWithFlags(&b->ready[i], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    lbm_batch_free(b);
    return LBM_ECUDA;
  }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int n) {
  if (!b || n < 0) return LBM_EINVAL;
  const long long t0 = b->h[0]->t;
  for (lbm* h : b->h) {
    if (((h->t - t0) & 1) != 0 || h->half || (h->ks->compact && !h->recs_valid)) return LBM_ESTATE;
    if (h->timed_out) return LBM_ETIMEOUT;
    if (h->unstable) return LBM_EUNSTABLE;
  }
  // the batch stream first waits for whatever each handle's own stream has queued ...
  for (size_t i = 0; i < b->h.size(); ++i) {
    if (b->h[i]->stream == b->stream) continue;
    if (cudaEventRecord(b->ready[i], b->h[i]->stream) != cudaSuccess ||
        cudaStreamWaitEvent(b->stream, b->ready[i], 0) != cudaSuccess)
      return LBM_ECUDA;
  }
  for (lbm* h : b->h) {
    lbm_status st = ensure_fix(h, b->stream);
    if (st != LBM_OK) return st;
    if (h->ks->compact) h->dens_ready = false;
  }
  int k = 0;
  if (n >= kGraphSteps) {
    const int parity = (int)(t0 & 1);
    if (!b->graph[parity]) {
      lbm_status st = batch_build(b, parity);
      if (st != LBM_OK) return st;
    }
    for (; k + kGraphSteps <= n; k += kGraphSteps) {
      if (cudaGraphLaunch(b->graph[parity], b->stream) != cudaSuccess) return LBM_ECUDA;
      for (lbm* h : b->h) {
        h->t += kGraphSteps;
        h->launches += h->graph_kernels[parity];
      }
    }
  }
  // the graph runs on the batch stream; later single steps of each handle go on that stream too
  if (k < n)
    for (lbm* h : b->h) {
      lbm_status st = enqueue_run(h, h->t, n - k, b->stream);
      if (st != LBM_OK) return st;
      h->t += n - k;
    }
  // ... and each handle's stream then waits for the batch, so later per-handle calls stay in order
  if (cudaEventRecord(b->done, b->stream) != cudaSuccess) return LBM_ECUDA;
  for (lbm* h : b->h)
    if (h->stream != b->stream && cudaStreamWaitEvent(h->stream, b->done, 0) != cudaSuccess) return LBM_ECUDA;
  return LBM_OK;
}

lbm_status lbm_batch_synchronize(lbm_batch* b) {
  if (!b) return LBM_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LBM_ECUDA;
  lbm_status worst = LBM_OK;
  for (lbm* h : b->h) {
    lbm_status st = lbm_synchronize(h);
    if (st != LBM_OK) worst = st;
  }
  return worst;
}

void lbm_batch_free(lbm_batch* b) {
  if (!b) return;
  batch_drop(b);
  for (auto s : b->branch)
    if (s) cudaStreamDestroy(s);
  for (auto e : b->ready)
    if (e) cudaEventDestroy(e);
  if (b->done) cudaEventDestroy(b->done);
  if (b->root) cudaStreamDestroy(b->root);
  delete b;
}

}  // extern "C"
