// C ABI of the batched analyses: plan (work lists, workspace layout, twiddle
// tables), autotuner (CTA size and line-FFT schedule per pass, chosen by
// timing the candidates on scratch data of the batch's shapes), and the
// analysis itself, replayed as one CUDA graph.
//
// Analyses of at least kBigPoints grid points run through the single-analysis
// passes (one plan each, whose pipelined row and column kernels move their
// bytes at several times the rate of the persistent batched passes); they are
// issued on kLanes streams that branch off the capture (largest first, each to
// the lane with the least work so far), beside the seven persistent launches
// that take every smaller analysis, so that the branches fill the GPU together.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/fftenkf.h"
#include "batch.cuh"
#include "k_batch.cuh"

using namespace fftenkf;

namespace fftenkf {
int sm_count();
void set_last_error(const std::string& msg);
}  // namespace fftenkf

namespace {
fftenkf_status bfail(fftenkf_status s, const std::string& m) {
  set_last_error(m);
  return s;
}
size_t rup(size_t x, size_t a) { return (x + a - 1) / a * a; }
const int kCandBt[2] = {128, 256};
#ifndef FFTENKF_BATCH_BIG_POINTS
#define FFTENKF_BATCH_BIG_POINTS (512LL * 256)
#endif
#ifndef FFTENKF_BATCH_LANES
#define FFTENKF_BATCH_LANES 8
#endif
constexpr long long kBigPoints = FFTENKF_BATCH_BIG_POINTS;   // grid points from which an analysis takes its own plan
constexpr int kLanes = FFTENKF_BATCH_LANES;
}  // namespace

struct fftenkf_batch_s {
  int count = 0, storage = 0;
  std::vector<BatchItem> items;              // host copy (pointers of the last bound call)
  BatchItem* d_items = nullptr;
  float2* d_tw = nullptr;
  int* d_status = nullptr;
  size_t ws_bytes = 0;
  void* own_ws = nullptr;
  std::vector<size_t> off_mean, off_A, off_W, off_chat, off_gain;
  // per-pass launch configuration
  int bt[kBPassCount], vsel[kBPassCount];
  BatchUnit* d_units[kBPassCount] = {};
  int n_units[kBPassCount] = {};
  size_t smem[kBPassCount] = {};
  int grid[kBPassCount] = {};
  // analyses on their own plans (null: in the batched passes), their workspace regions
  std::vector<fftenkf_plan> sub;
  std::vector<size_t> off_sub;
  cudaStream_t lane[kLanes] = {};
  cudaEvent_t ev_fork = nullptr, ev_lane[kLanes] = {};
  // graph of the launches
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  char* bound_ws = nullptr;
  bool items_dirty = true;
  bool sub_dirty = true;   // pointers of a planned analysis changed: capture again
};

// work list and launch shape of pass `pass` for CTA size bt and schedule vsel
static fftenkf_status build_pass(fftenkf_batch b, int pass, int bt, int vsel) {
  struct U {
    double cost;
    BatchUnit u;
  };
  std::vector<U> list;
  size_t smem = 0;
  for (int i = 0; i < b->count; ++i) {
    if (b->sub[i]) continue;   // on its own plan
    const BatchItem& it = b->items[i];
    const int n = batch_units(pass, it, bt, vsel);
    const double c = batch_unit_cost(pass, it, bt, vsel);
    for (int u = 0; u < n; ++u) list.push_back({c, {i, u}});
    smem = std::max(smem, batch_smem(pass, it, bt, vsel));
  }
  if (smem > 200 * 1024) return bfail(FFTENKF_EUNSUPPORTED, "batched unit exceeds shared memory");
  std::stable_sort(list.begin(), list.end(), [](const U& a, const U& c) { return a.cost > c.cost; });
  std::vector<BatchUnit> units(list.size());
  for (size_t i = 0; i < list.size(); ++i) units[i] = list[i].u;
  if (b->d_units[pass]) cudaFree(b->d_units[pass]);
  b->d_units[pass] = nullptr;
  if (!units.empty()) {
    if (cudaMalloc(&b->d_units[pass], units.size() * sizeof(BatchUnit)) != cudaSuccess)
      return bfail(FFTENKF_ENOMEM, "work list allocation failed");
    cudaMemcpy(b->d_units[pass], units.data(), units.size() * sizeof(BatchUnit), cudaMemcpyHostToDevice);
  }
  b->n_units[pass] = (int)units.size();
  b->bt[pass] = (pass == kBGain) ? 256 : bt;
  b->vsel[pass] = vsel;
  b->smem[pass] = smem;
  // persistent grid: as many CTAs as fit on the GPU at this shared memory size
  const int by_smem = smem ? (int)((220 * 1024) / (smem + 1024)) : 16;
  int per_sm = std::max(1, std::min(by_smem, 2048 / b->bt[pass]));
  b->grid[pass] = std::max(1, std::min((int)units.size(), sm_count() * per_sm));
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return FFTENKF_OK;
}

static BatchParams pass_params(fftenkf_batch b, int pass) {
  BatchParams p;
  p.items = b->d_items;
  p.units = b->d_units[pass];
  p.n_units = b->n_units[pass];
  p.storage = b->storage;
  p.mode = (pass == kBRowInnov) ? kInnovation : kAnomaly;
  p.vsel = b->vsel[pass];
  p.status = b->d_status;
  return p;
}

static cudaError_t run_passes(fftenkf_batch b, cudaStream_t s) {
  for (int pass = 0; pass < kBPassCount; ++pass) {
    if (b->n_units[pass] == 0) continue;   // every analysis on its own plan
    cudaError_t e = launch_batch_pass(pass, pass_params(b, pass), b->bt[pass], b->smem[pass], b->grid[pass], s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The whole batch on stream s: the planned analyses on the lanes (forked from s and joined
// back), the persistent passes of the others on s.
static fftenkf_status run_all(fftenkf_batch b, void* const* ens, const float* const* data, const void* const* pert,
                              const double* const* rhat, char* ws, cudaStream_t s) {
  bool any = false;
  for (int i = 0; i < b->count; ++i) any |= b->sub[i] != nullptr;
  cudaError_t e = cudaSuccess;
  if (any) {
    e = cudaEventRecord(b->ev_fork, s);
    for (int l = 0; l < kLanes && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(b->lane[l], b->ev_fork, 0);
    if (e != cudaSuccess) return bfail(FFTENKF_ECUDA, std::string("fork: ") + cudaGetErrorString(e));
    std::vector<int> order;
    for (int i = 0; i < b->count; ++i)
      if (b->sub[i]) order.push_back(i);
    auto cost = [&](int i) { return (double)b->items[i].N * b->items[i].ny * b->items[i].nx; };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
    double load[kLanes] = {};
    for (int i : order) {
      int l = 0;
      for (int q = 1; q < kLanes; ++q)
        if (load[q] < load[l]) l = q;
      load[l] += cost(i);
      fftenkf_status st = fftenkf_analyze(b->sub[i], ens[i], data[i], pert[i], rhat[i], nullptr, ws + b->off_sub[i],
                                          b->lane[l]);
      if (st != FFTENKF_OK) return st;
    }
  }
  e = run_passes(b, s);
  if (e != cudaSuccess) return bfail(FFTENKF_ECUDA, std::string("batched passes: ") + cudaGetErrorString(e));
  if (any) {
    for (int l = 0; l < kLanes && e == cudaSuccess; ++l) {
      e = cudaEventRecord(b->ev_lane[l], b->lane[l]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_lane[l], 0);
    }
    if (e != cudaSuccess) return bfail(FFTENKF_ECUDA, std::string("join: ") + cudaGetErrorString(e));
  }
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_plan_batched(fftenkf_batch* out, int count, const fftenkf_dims* dims) {
  set_last_error("");
  if (!out || !dims || count <= 0) return bfail(FFTENKF_EINVAL, "null argument or empty batch");
  *out = nullptr;
  const int storage = dims[0].storage;
  for (int i = 0; i < count; ++i) {
    const fftenkf_dims& d = dims[i];
    if (d.n_blocks != 1) return bfail(FFTENKF_EUNSUPPORTED, "batched analyses have one (observed) block each");
    if (d.storage != storage) return bfail(FFTENKF_EINVAL, "all batched analyses share one storage type");
    if (d.storage != FFTENKF_F32 && d.storage != FFTENKF_BF16) return bfail(FFTENKF_EINVAL, "unknown storage");
    if (d.n_members < 2) return bfail(FFTENKF_EUNSUPPORTED, "need at least 2 members");
    if (d.nx % 2 || !batch_line_supported(d.nx / 2) || !batch_line_supported(d.ny))
      return bfail(FFTENKF_EUNSUPPORTED, "batched sizes: ny and nx/2 in {2^a, 3*2^a} between 16 and 1024");
  }
  fftenkf_batch b = new fftenkf_batch_s();
  b->count = count;
  b->storage = storage;
  b->items.resize(count);
  // twiddle tables, one set per distinct line length
  std::vector<float2> tw;
  std::map<int, size_t> off_stage[2];
  std::map<int, size_t> off_x;
  auto stage_table = [&](int n, int sel) {
    if (off_stage[sel].count(n)) return;
    off_stage[sel][n] = tw.size();
    const int V = plan_V(n, sel);
    for (int i = 0; i < twiddle_count(n, V); ++i) {
      const double ang = 2.0 * M_PI * (double)twiddle_exponent(n, V, i) / (double)n;
      tw.push_back(make_float2((float)std::cos(ang), (float)-std::sin(ang)));
    }
    if (tw.size() % 2) tw.push_back(make_float2(0.f, 0.f));
  };
  for (int i = 0; i < count; ++i) {
    const int L = dims[i].nx / 2, ny = dims[i].ny;
    for (int sel = 0; sel < 2; ++sel) {
      stage_table(L, sel);
      stage_table(ny, sel);
    }
    if (!off_x.count(dims[i].nx)) {
      off_x[dims[i].nx] = tw.size();
      for (int k = 0; k <= L; ++k) {
        const double ang = 2.0 * M_PI * (double)k / (double)dims[i].nx;
        tw.push_back(make_float2((float)std::cos(ang), (float)-std::sin(ang)));
      }
      if (tw.size() % 2) tw.push_back(make_float2(0.f, 0.f));
    }
  }
  cudaError_t e = cudaMalloc(&b->d_tw, tw.size() * sizeof(float2));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_items, count * sizeof(BatchItem));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  for (int l = 0; l < kLanes && e == cudaSuccess; ++l) {
    e = cudaStreamCreateWithFlags(&b->lane[l], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_lane[l], cudaEventDisableTiming);
  }
  b->sub.assign(count, nullptr);
  b->off_sub.assign(count, 0);
  if (e != cudaSuccess) {
    fftenkf_batch_destroy(b);
    return bfail(FFTENKF_ENOMEM, "batched plan allocation failed");
  }
  // analyses large enough to fill the GPU through their own passes get a plan each; a shape
  // the single-analysis plan does not take stays in the batched passes
  for (int i = 0; i < count; ++i) {
    if ((long long)dims[i].ny * dims[i].nx < kBigPoints) continue;
    fftenkf_dims d = dims[i];
    const uint8_t observed = 1;
    fftenkf_plan sp = nullptr;
    if (fftenkf_plan_create(&sp, &d, &observed) == FFTENKF_OK) b->sub[i] = sp;
  }
  set_last_error("");
  // workspace layout, item shapes and twiddle pointers
  size_t off = 0;
  b->off_mean.resize(count);
  b->off_A.resize(count);
  b->off_W.resize(count);
  b->off_chat.resize(count);
  b->off_gain.resize(count);
  for (int i = 0; i < count; ++i) {
    BatchItem& it = b->items[i];
    memset(&it, 0, sizeof(it));
    it.ny = dims[i].ny;
    it.nx = dims[i].nx;
    it.L = it.nx / 2;
    it.N = dims[i].n_members;
    const size_t G = (size_t)it.ny * it.nx, line = (size_t)it.L * it.ny * sizeof(float2);
    const size_t tab = (size_t)(it.L + 1) * it.ny * sizeof(float);
    it.twL = b->d_tw + off_stage[0][it.L];
    it.twL_alt = b->d_tw + off_stage[1][it.L];
    it.twY = b->d_tw + off_stage[0][it.ny];
    it.twY_alt = b->d_tw + off_stage[1][it.ny];
    it.twX = b->d_tw + off_x[it.nx];
    if (b->sub[i]) {   // the plan's workspace instead of the batched regions
      size_t sb = 0;
      fftenkf_workspace_size(b->sub[i], &sb);
      b->off_sub[i] = off; off = rup(off + sb, 256);
      b->off_mean[i] = b->off_A[i] = b->off_W[i] = b->off_chat[i] = b->off_gain[i] = b->off_sub[i];
      continue;
    }
    b->off_mean[i] = off; off = rup(off + G * sizeof(float), 256);
    b->off_A[i] = off;    off = rup(off + it.N * line, 256);
    b->off_W[i] = off;    off = rup(off + it.N * line, 256);
    b->off_chat[i] = off; off = rup(off + tab, 256);
    b->off_gain[i] = off; off = rup(off + tab, 256);
  }
  b->ws_bytes = off;
  for (int pass = 0; pass < kBPassCount; ++pass) {
    fftenkf_status st = build_pass(b, pass, 256, 0);
    if (st != FFTENKF_OK) {
      fftenkf_batch_destroy(b);
      return st;
    }
  }
  *out = b;
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_batch_destroy(fftenkf_batch b) {
  if (!b) return FFTENKF_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (fftenkf_plan sp : b->sub)
    if (sp) fftenkf_plan_destroy(sp);
  for (int l = 0; l < kLanes; ++l) {
    if (b->lane[l]) cudaStreamDestroy(b->lane[l]);
    if (b->ev_lane[l]) cudaEventDestroy(b->ev_lane[l]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  for (int p = 0; p < kBPassCount; ++p)
    if (b->d_units[p]) cudaFree(b->d_units[p]);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_tw) cudaFree(b->d_tw);
  if (b->d_status) cudaFree(b->d_status);
  if (b->own_ws) cudaFree(b->own_ws);
  delete b;
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_batch_workspace_size(fftenkf_batch b, size_t* bytes) {
  if (!b || !bytes) return bfail(FFTENKF_EINVAL, "null argument");
  *bytes = b->ws_bytes;
  return FFTENKF_OK;
}

static fftenkf_status bind(fftenkf_batch b, void* const* ens, const float* const* data, const void* const* pert,
                           const double* const* rhat, char* ws) {
  bool changed = (ws != b->bound_ws);
  for (int i = 0; i < b->count; ++i) {
    if (!ens[i] || !data[i] || !pert[i] || !rhat[i]) return bfail(FFTENKF_EINVAL, "null item pointer");
    if (((uintptr_t)ens[i] | (uintptr_t)data[i] | (uintptr_t)pert[i] | (uintptr_t)rhat[i]) % 16)
      return bfail(FFTENKF_EINVAL, "item pointers must be 16-byte aligned");
    BatchItem& it = b->items[i];
    const bool moved = it.ens != ens[i] || it.data != data[i] || it.pert != pert[i] || it.rhat != rhat[i];
    changed |= moved;
    if (b->sub[i] && moved) b->sub_dirty = true;   // its kernels take the pointers by value
    it.ens = ens[i];
    it.data = data[i];
    it.pert = pert[i];
    it.rhat = rhat[i];
    it.mean = reinterpret_cast<float*>(ws + b->off_mean[i]);
    it.A = reinterpret_cast<float2*>(ws + b->off_A[i]);
    it.W = reinterpret_cast<float2*>(ws + b->off_W[i]);
    it.chat = reinterpret_cast<float*>(ws + b->off_chat[i]);
    it.gain = reinterpret_cast<float*>(ws + b->off_gain[i]);
  }
  if (ws != b->bound_ws) b->sub_dirty = true;
  b->bound_ws = ws;
  b->items_dirty |= changed;
  return FFTENKF_OK;
}

static fftenkf_status batch_ws(fftenkf_batch b, void* workspace, char** ws) {
  if (workspace) {
    if ((uintptr_t)workspace % 256) return bfail(FFTENKF_EINVAL, "workspace must be 256-byte aligned");
    *ws = static_cast<char*>(workspace);
    return FFTENKF_OK;
  }
  if (!b->own_ws && cudaMalloc(&b->own_ws, b->ws_bytes) != cudaSuccess) {
    b->own_ws = nullptr;
    return bfail(FFTENKF_ENOMEM, "workspace allocation failed");
  }
  *ws = static_cast<char*>(b->own_ws);
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_analyze_batched(fftenkf_batch b, void* const* ensembles, const float* const* data,
                                                  const void* const* perturbations, const double* const* rhat,
                                                  void* workspace, void* stream) {
  set_last_error("");
  if (!b || !ensembles || !data || !perturbations || !rhat) return bfail(FFTENKF_EINVAL, "null argument");
  char* ws;
  fftenkf_status st = batch_ws(b, workspace, &ws);
  if (st != FFTENKF_OK) return st;
  st = bind(b, ensembles, data, perturbations, rhat, ws);
  if (st != FFTENKF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (b->items_dirty) {
    // pageable copy: the runtime stages the host table before returning, ordered on s
    e = cudaMemcpyAsync(b->d_items, b->items.data(), b->count * sizeof(BatchItem), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bfail(FFTENKF_ECUDA, std::string("item table: ") + cudaGetErrorString(e));
    b->items_dirty = false;
  }
  if (b->exec && b->sub_dirty) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (!b->exec) {
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    fftenkf_status rs = FFTENKF_OK;
    std::string rmsg;
    if (e == cudaSuccess) {
      rs = run_all(b, ensembles, data, perturbations, rhat, ws, b->cap);
      if (rs != FFTENKF_OK) rmsg = fftenkf_last_error();
      e = cudaStreamEndCapture(b->cap, &g);
    }
    if (rs != FFTENKF_OK) {
      if (g) cudaGraphDestroy(g);
      return bfail(rs, "graph capture: " + rmsg);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      return bfail(FFTENKF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    b->sub_dirty = false;
  }
  e = cudaGraphLaunch(b->exec, s);
  if (e != cudaSuccess) return bfail(FFTENKF_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  return FFTENKF_OK;
}

// Time every (CTA size, schedule) candidate of every pass on zero-filled
// scratch inputs of the batch's shapes and keep the fastest.  Allocates the
// scratch inputs (one ensemble's worth per item) for the duration of the call.
extern "C" fftenkf_status fftenkf_batch_autotune(fftenkf_batch b, void* workspace, void* stream, double* best_ms) {
  set_last_error("");
  if (!b) return bfail(FFTENKF_EINVAL, "null argument");
  char* ws;
  fftenkf_status st = batch_ws(b, workspace, &ws);
  if (st != FFTENKF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int es = b->storage == FFTENKF_BF16 ? 2 : 4;
  size_t bytes = 0;
  std::vector<size_t> oe(b->count), od(b->count), op(b->count), orh(b->count);
  for (int i = 0; i < b->count; ++i) {
    const BatchItem& it = b->items[i];
    const size_t G = (size_t)it.ny * it.nx;
    oe[i] = bytes; bytes = rup(bytes + it.N * G * es, 256);
    od[i] = bytes; bytes = rup(bytes + G * 4, 256);
    op[i] = bytes; bytes = rup(bytes + it.N * G * es, 256);
    orh[i] = bytes; bytes = rup(bytes + (size_t)it.ny * (it.L + 1) * 8, 256);
  }
  char* scratch = nullptr;
  if (cudaMalloc(&scratch, bytes) != cudaSuccess) return bfail(FFTENKF_ENOMEM, "autotune scratch allocation failed");
  cudaMemsetAsync(scratch, 0, bytes, s);
  std::vector<void*> ens(b->count), pert(b->count);
  std::vector<const float*> dat(b->count);
  std::vector<const double*> rh(b->count);
  for (int i = 0; i < b->count; ++i) {
    ens[i] = scratch + oe[i];
    dat[i] = reinterpret_cast<const float*>(scratch + od[i]);
    pert[i] = scratch + op[i];
    rh[i] = reinterpret_cast<const double*>(scratch + orh[i]);
  }
  std::vector<BatchItem> saved = b->items;
  char* saved_ws = b->bound_ws;
  bind(b, ens.data(), dat.data(), pert.data(), rh.data(), ws);
  cudaMemcpyAsync(b->d_items, b->items.data(), b->count * sizeof(BatchItem), cudaMemcpyHostToDevice, s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double total = 0.0;
  for (int pass = 0; pass < kBPassCount && st == FFTENKF_OK; ++pass) {
    float best = 1e30f;
    int bbt = 256, bvs = 0;
    const int nv = (pass == kBMean || pass == kBGain) ? 1 : 2;
    const int nb = (pass == kBGain) ? 1 : 2;
    for (int ci = 0; ci < nb; ++ci)
      for (int vs = 0; vs < nv; ++vs) {
        if (build_pass(b, pass, kCandBt[ci], vs) != FFTENKF_OK) continue;
        const BatchParams p = pass_params(b, pass);
        float ms = 0.f;
        for (int rep = 0; rep < 3; ++rep) {   // first repetition warms up
          cudaEventRecord(e0, s);
          launch_batch_pass(pass, p, b->bt[pass], b->smem[pass], b->grid[pass], s);
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float t = 0.f;
          cudaEventElapsedTime(&t, e0, e1);
          if (rep) ms += t;
        }
        if (ms < best) {
          best = ms;
          bbt = kCandBt[ci];
          bvs = vs;
        }
      }
    st = build_pass(b, pass, bbt, bvs);
    total += best / 2.0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t e = cudaStreamSynchronize(s);
  cudaMemset(b->d_status, 0, sizeof(int));
  cudaFree(scratch);
  b->items = saved;
  b->bound_ws = saved_ws;
  b->items_dirty = true;
  if (best_ms) *best_ms = total;
  if (e != cudaSuccess) return bfail(FFTENKF_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
  return st;
}

extern "C" fftenkf_status fftenkf_batch_schedule(fftenkf_batch b, int* cta_threads, int* sched, int n) {
  if (!b || !cta_threads || !sched) return bfail(FFTENKF_EINVAL, "null argument");
  for (int p = 0; p < kBPassCount && p < n; ++p) {
    cta_threads[p] = b->bt[p];
    sched[p] = b->vsel[p];
  }
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_batch_last_device_status(fftenkf_batch b, void* stream) {
  if (!b) return bfail(FFTENKF_EINVAL, "null argument");
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return bfail(FFTENKF_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
  int word = 0;
  e = cudaMemcpy(&word, b->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return bfail(FFTENKF_ECUDA, std::string("status word: ") + cudaGetErrorString(e));
  fftenkf_status worst = FFTENKF_OK;
  for (fftenkf_plan sp : b->sub) {   // the analyses on their own plans
    if (!sp) continue;
    const fftenkf_status st = fftenkf_last_device_status(sp, stream);
    if (st != FFTENKF_OK && worst == FFTENKF_OK) worst = st;
  }
  if (word & kStatusNonFinite) return bfail(FFTENKF_ENONFINITE, "non-finite spectral covariance");
  if (worst != FFTENKF_OK) return bfail(worst, "an analysis on its own plan: " + std::string(fftenkf_last_error()));
  return FFTENKF_OK;
}
