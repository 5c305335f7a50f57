// C ABI: plans, argument validation and the order of the passes.
//
// analyze (Sec. 2.1, eq. spectral-multi-enkf), on the caller's stream unless noted:
//   0. rhat_transpose  rhat to the column layout            [auxiliary stream, overlaps 2]
//   2. row_fwd anomaly  rows of F(u_k^(j) - u_0^(j)), k >= 1, and of sqrt(N) F(ubar^(j) - u_0^(j))
//                      in the place of k = 0 -> A (first member as pivot: no mean pass)
//   3. col_stats       columns of F, chat^(oo), chat^(jo) and the gains
//                      chat/(chat^(oo)+rhat) -> goo, gjo (eq. dii, cov-multi-spectral, spectral-multi-enkf)
//   5. row_fwd innov   rows of F(d_o + e_{k,o} - u_k^(o)) -> W
//   6. col_update      gain x innovation, inverse columns -> S (aliases A)
//   7. row_inv         inverse rows, u_k^(j) += increment
// With a caller-supplied spectrum, 1-3 are skipped and the gain pass (4) reads the
// tables on the auxiliary stream, overlapping 5.
// When the fused column pass covers the plan (one or two observed blocks, not coupled, the
// wide column schedule), steps 3 and 6 are one launch after step 5:
//   5. row_fwd innov, 3+6. col_fused (columns of F, chat, gains, gain x innovation, inverse
//   columns -> S), 7. row_inv.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fftenkf.h"
#include "common.cuh"

using namespace fftenkf;

// kPassMean: the retired mean pass (the anomaly rows take the first member as pivot); its slot
// keeps the later indices stable and its time reads 0
enum Pass { kPassMean, kPassRowAnom, kPassStats, kPassGain, kPassRowInnov, kPassUpdate, kPassRowInv,
            kPassChatOut, kPassRhatT, kPassFused, kPassCount };
static const char* kPassNames[kPassCount] = {"mean", "row_fwd_anomaly", "col_stats", "gain",
                                             "row_fwd_innovation", "col_update", "row_inv", "chat_out",
                                             "rhat_transpose", "col_fused"};

namespace {
thread_local std::string g_last_error;

fftenkf_status fail(fftenkf_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}
fftenkf_status cuda_fail(cudaError_t e, const char* where) {
  return fail(FFTENKF_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
bool is_line(int n) { return line_supported(n); }
bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
}  // namespace

namespace fftenkf {
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace fftenkf

struct fftenkf_plan_s {
  int ny, nx, L, M, N, storage;
  int n_obs, n_un;
  int obs[kMaxObs];
  int un[kMaxBlocks];
  int obs_of_block[kMaxBlocks];
  int un_of_block[kMaxBlocks];
  float2* d_tw = nullptr;     // [L] row twiddles, [ny] column twiddles, [L+1] real-FFT twiddles
  float4* d_tw4 = nullptr;    // paired column twiddles of the fused column pass, both schedules
  size_t off_tw4[2] = {0, 0};
  bool fused_ok[2] = {false, false};   // the fused column pass covers the plan with schedule 0 / 1
  int* d_status = nullptr;
  cudaStream_t aux = nullptr;
  bool coupled = false;   // observed blocks coupled through their cross-covariance (n_obs <= 2)
  int n_pair = 0;         // observed-pair tables in the column statistics (coupled: n_obs (n_obs-1) / 2)
  // tensor map of the increment spectra for the inverse row pass, cached for one workspace
  alignas(64) CUtensorMap tm;
  float2* tm_S = nullptr;
  int tm_R = 0;
  bool tm_ok = false;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // workspace layout (byte offsets)
  size_t off_A, off_W, off_chat, off_goo, off_gjo, off_rhat_t, off_amp, ws_bytes;
  void* own_ws = nullptr;
  int device = 0;
  // per-pass CUDA-event timing (fftenkf_set_profiling); a ring of event pairs per pass
  bool prof = false;
  static constexpr int kSlots = 64;
  cudaEvent_t ev[kPassCount][kSlots][2] = {};
  int used[kPassCount] = {};
  double acc_ms[kPassCount] = {};
  int launches[kPassCount] = {};
  size_t off_twL[2] = {0, 0}, off_twY[2] = {0, 0}, off_twX = 0;
  int sched[kPassCount] = {};   // line-FFT schedule (plan_V selector) per pass
  int expire_first_wait = 0;    // test setting (fftenkf_set_expire_first_wait)
  const float2* twL(int sel) const { return d_tw + off_twL[sel]; }
  const float2* twY(int sel) const { return d_tw + off_twY[sel]; }
  const float2* twX() const { return d_tw + off_twX; }
  // the fused column pass runs when it covers the plan and the column schedules are the wide ones
  bool use_fused() const {
    return fused_ok[sched[kPassFused] & 1] && !coupled && sched[kPassStats] == 0 && sched[kPassUpdate] == 0;
  }
};

// fold a completed slot into the totals
static void prof_drain(fftenkf_plan p, int pass, int slot) {
  float ms = 0.f;
  cudaEventSynchronize(p->ev[pass][slot][1]);
  if (cudaEventElapsedTime(&ms, p->ev[pass][slot][0], p->ev[pass][slot][1]) == cudaSuccess) {
    p->acc_ms[pass] += ms;
    p->launches[pass] += 1;
  }
}
static void prof_begin(fftenkf_plan p, int pass, cudaStream_t s) {
  if (!p->prof) return;
  int slot = p->used[pass] % fftenkf_plan_s::kSlots;
  if (p->used[pass] >= fftenkf_plan_s::kSlots) prof_drain(p, pass, slot);
  if (!p->ev[pass][slot][0]) {
    cudaEventCreate(&p->ev[pass][slot][0]);
    cudaEventCreate(&p->ev[pass][slot][1]);
  }
  cudaEventRecord(p->ev[pass][slot][0], s);
}
static void prof_end(fftenkf_plan p, int pass, cudaStream_t s) {
  if (!p->prof) return;
  int slot = p->used[pass] % fftenkf_plan_s::kSlots;
  cudaEventRecord(p->ev[pass][slot][1], s);
  p->used[pass] += 1;
}

static float2 unit_root(long long e, long long n) {   // exp(-2 pi i e / n), FP64 then rounded
  const double ang = 2.0 * M_PI * (double)(e % n) / (double)n;
  return make_float2((float)std::cos(ang), (float)-std::sin(ang));
}

// plain table exp(-2 pi i e / n), e < count
static void host_twiddles(std::vector<float2>& out, int n, int count) {
  for (int e = 0; e < count; ++e) out.push_back(unit_root(e, n));
}

// stage-major table of the line FFT plan (n, V), laid out as fft_core.cuh reads it
static void host_stage_twiddles(std::vector<float2>& out, int n, int V) {
  const int count = twiddle_count(n, V);
  for (int i = 0; i < count; ++i) out.push_back(unit_root(twiddle_exponent(n, V, i), n));
}

// covariance tables per wavenumber in the column statistics
static int table_floats(const fftenkf_plan_s* p) { return p->n_obs + 2 * p->n_pair + 2 * p->n_obs * p->n_un; }

// workspace layout (byte offsets); the gain region holds goo/gjo, or gall [M][n_obs] (complex) when coupled
static void layout(fftenkf_plan_s* p) {
  const size_t G = (size_t)p->ny * p->nx;
  const size_t line = (size_t)p->L * p->ny * sizeof(float2);     // one field's row spectra
  const size_t tab = (size_t)(p->L + 1) * p->ny;
  const size_t gain_tables = p->coupled ? (size_t)p->M * p->n_obs : (size_t)p->n_obs * p->n_un;
  size_t off = 0;
  p->off_A = off;    off = round_up(off + (size_t)p->M * p->N * line, 256);
  p->off_chat = off; off = round_up(off + (size_t)table_floats(p) * tab * sizeof(float), 256);
  p->off_W = off;    off = round_up(off + (size_t)p->N * p->n_obs * line, 256);
  p->off_goo = off;  off = round_up(off + (size_t)p->n_obs * tab * sizeof(float), 256);
  p->off_gjo = off;  off = round_up(off + gain_tables * tab * sizeof(float2), 256);
  p->off_rhat_t = off; off = round_up(off + (size_t)p->n_obs * tab * sizeof(double), 256);
  p->off_amp = off;  off = round_up(off + (size_t)p->n_obs * tab * sizeof(float), 256);
  p->ws_bytes = off;
}

extern "C" fftenkf_status fftenkf_plan_create(fftenkf_plan* plan, const fftenkf_dims* dims,
                                              const uint8_t* observed_mask) {
  g_last_error.clear();
  if (!plan || !dims || !observed_mask) return fail(FFTENKF_EINVAL, "null argument");
  *plan = nullptr;
  const fftenkf_dims d = *dims;
  if (d.ny <= 0 || d.nx <= 0 || d.n_blocks <= 0 || d.n_members <= 0)
    return fail(FFTENKF_EINVAL, "dimensions must be positive");
  if (d.storage != FFTENKF_F32 && d.storage != FFTENKF_BF16) return fail(FFTENKF_EINVAL, "unknown storage");
  if (d.n_members < 2) return fail(FFTENKF_EUNSUPPORTED, "need at least 2 members (eq. dii divides by N-1)");
  if (d.n_blocks > kMaxBlocks) return fail(FFTENKF_EUNSUPPORTED, "at most 16 blocks");
  if (d.nx % 2 || !row_line_supported(d.nx / 2) || d.nx < 16 || d.nx > 8192)
    return fail(FFTENKF_EUNSUPPORTED, "nx must be 2^a or 3*2^a in [16, 8192]");
  if (!is_line(d.ny) || d.ny < 16 || d.ny > 4096)
    return fail(FFTENKF_EUNSUPPORTED, "ny must be 2^a or 3*2^a in [16, 4096]");
  fftenkf_plan_s* p = new fftenkf_plan_s();
  p->ny = d.ny;
  p->nx = d.nx;
  p->L = d.nx / 2;
  p->M = d.n_blocks;
  p->N = d.n_members;
  p->storage = d.storage;
  p->n_obs = p->n_un = 0;
  for (int j = 0; j < p->M; ++j) {
    p->obs_of_block[j] = p->un_of_block[j] = -1;
    if (observed_mask[j]) {
      if (p->n_obs >= kMaxObs) {
        delete p;
        return fail(FFTENKF_EUNSUPPORTED, "at most 4 observed blocks");
      }
      p->obs_of_block[j] = p->n_obs;
      p->obs[p->n_obs++] = j;
    } else {
      p->un_of_block[j] = p->n_un;
      p->un[p->n_un++] = j;
    }
  }
  const int nf = p->n_obs + 2 * p->n_obs * p->n_un;
  if (p->n_obs > 0 && (col_stats_smem(p->ny, nf, 0, nullptr) == 0 || col_update_smem(p->ny, p->n_obs, 0, nullptr, nullptr) == 0)) {
    delete p;
    return fail(FFTENKF_EUNSUPPORTED, "covariance tables per column exceed shared memory (reduce blocks or ny)");
  }
  layout(p);
  cudaGetDevice(&p->device);
  std::vector<float2> tw;
  for (int sel = 0; sel < 2; ++sel) {
    p->off_twL[sel] = tw.size();
    host_stage_twiddles(tw, p->L, plan_V(p->L, sel));
    p->off_twY[sel] = tw.size();
    host_stage_twiddles(tw, p->ny, plan_V(p->ny, sel));
  }
  p->off_twX = tw.size();
  host_twiddles(tw, p->nx, p->L + 1);
  if (tw.size() % 2) tw.push_back(make_float2(0.f, 0.f));
  cudaError_t e = cudaMalloc(&p->d_tw, tw.size() * sizeof(float2));
  if (e != cudaSuccess) {
    delete p;
    return fail(FFTENKF_ENOMEM, "twiddle allocation failed");
  }
  e = cudaMemcpy(p->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
  std::vector<float4> t4;
  for (int sel = 0; sel < 2; ++sel) {
    p->fused_ok[sel] = col_fused_supported(p->ny, p->n_obs, p->M, sel);
    if (!p->fused_ok[sel]) continue;
    std::vector<float2> t1;
    host_stage_twiddles(t1, p->ny, plan_V(p->ny, sel));
    p->off_tw4[sel] = t4.size();
    for (const float2& w : t1) t4.push_back(make_float4(w.x, w.x, w.y, w.y));
    t4.push_back(make_float4(0.f, 0.f, 0.f, 0.f));
  }
  if (e == cudaSuccess && !t4.empty()) {
    e = cudaMalloc(&p->d_tw4, t4.size() * sizeof(float4));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_tw4, t4.data(), t4.size() * sizeof(float4), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMalloc(&p->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    fftenkf_plan_destroy(p);
    return cuda_fail(e, "plan_create");
  }
  *plan = p;
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_plan_destroy(fftenkf_plan p) {
  if (!p) return FFTENKF_OK;
  if (p->own_ws) cudaFree(p->own_ws);
  if (p->d_tw) cudaFree(p->d_tw);
  if (p->d_tw4) cudaFree(p->d_tw4);
  if (p->d_status) cudaFree(p->d_status);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->aux) cudaStreamDestroy(p->aux);
  for (int a = 0; a < kPassCount; ++a)
    for (int b = 0; b < fftenkf_plan_s::kSlots; ++b)
      for (int c = 0; c < 2; ++c)
        if (p->ev[a][b][c]) cudaEventDestroy(p->ev[a][b][c]);
  delete p;
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_workspace_size(fftenkf_plan p, size_t* bytes) {
  if (!p || !bytes) return fail(FFTENKF_EINVAL, "null argument");
  *bytes = p->ws_bytes;
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_spectrum_size(fftenkf_plan p, size_t* n) {
  if (!p || !n) return fail(FFTENKF_EINVAL, "null argument");
  const size_t K = (size_t)p->ny * (p->L + 1);
  const size_t n_cplx = p->coupled ? (size_t)p->n_obs * (p->M - 1) : (size_t)p->n_obs * p->n_un;
  *n = (size_t)p->n_obs * K + n_cplx * 2 * K;
  return FFTENKF_OK;
}

static fftenkf_status get_workspace(fftenkf_plan p, void* ws, char** out) {
  if (ws) {
    if (!aligned(ws, 256)) return fail(FFTENKF_EINVAL, "workspace must be 256-byte aligned");
    *out = static_cast<char*>(ws);
    return FFTENKF_OK;
  }
  if (!p->own_ws) {
    cudaError_t e = cudaMalloc(&p->own_ws, p->ws_bytes);
    if (e != cudaSuccess) {
      p->own_ws = nullptr;
      return fail(FFTENKF_ENOMEM, "workspace allocation failed");
    }
  }
  *out = static_cast<char*>(p->own_ws);
  return FFTENKF_OK;
}

static ColFusedParams fused_params(fftenkf_plan p, char* ws) {
  ColFusedParams f;
  memset(&f, 0, sizeof(f));
  f.ny = p->ny; f.L = p->L; f.M = p->M; f.N = p->N; f.n_obs = p->n_obs; f.n_un = p->n_un;
  for (int r = 0; r < p->M; ++r) f.role_block[r] = (r < p->n_obs) ? p->obs[r] : p->un[r - p->n_obs];
  f.A = reinterpret_cast<const float2*>(ws + p->off_A);
  f.S = reinterpret_cast<float2*>(ws + p->off_A);
  f.vsel = p->sched[kPassFused] & 1;
  f.tw = p->d_tw4 + p->off_tw4[f.vsel];
  f.scale = (float)(1.0 / ((double)(p->N - 1) * (double)p->ny * (double)p->nx));
  f.inv_G = (float)(1.0 / ((double)p->ny * (double)p->nx));
  f.status = p->d_status;
  return f;
}

// step 2: anomaly row spectra (pivot form) -> A
static cudaError_t run_anomaly_rows(fftenkf_plan p, const void* ens, char* ws, cudaStream_t s) {
  RowFwdParams rp;
  memset(&rp, 0, sizeof(rp));
  rp.ny = p->ny; rp.nx = p->nx; rp.L = p->L; rp.M = p->M; rp.N = p->N;
  rp.n_obs = p->n_obs; rp.mode = kAnomaly; rp.storage = p->storage;
  rp.ens = ens;
  rp.out = reinterpret_cast<float2*>(ws + p->off_A);
  rp.vsel = p->sched[kPassRowAnom];
  rp.twL = p->twL(rp.vsel & 1); rp.twX = p->twX(); rp.status = p->d_status;
  rp.expire_first_wait = p->expire_first_wait;
  prof_begin(p, kPassRowAnom, s);
  cudaError_t e = launch_row_fwd(rp, p->M * p->N, s);
  prof_end(p, kPassRowAnom, s);
  return e;
}

// steps 2-3: anomaly row spectra, column statistics -> chat_t
// with rhat_t != null the column pass also forms the gains (analysis) and skips chat_t
static cudaError_t run_statistics(fftenkf_plan p, const void* ens, char* ws, cudaStream_t s, const double* rhat_t,
                                  cudaEvent_t wait_before_stats = nullptr) {
  cudaError_t e = run_anomaly_rows(p, ens, ws, s);
  if (e != cudaSuccess) return e;
  ColStatsParams cp;
  memset(&cp, 0, sizeof(cp));
  cp.ny = p->ny; cp.L = p->L; cp.M = p->M; cp.N = p->N; cp.n_obs = p->n_obs; cp.n_un = p->n_un;
  for (int i = 0; i < p->n_obs; ++i) cp.obs[i] = p->obs[i];
  for (int u = 0; u < p->n_un; ++u) cp.un[u] = p->un[u];
  cp.A = reinterpret_cast<const float2*>(ws + p->off_A);
  cp.chat = rhat_t ? nullptr : reinterpret_cast<float*>(ws + p->off_chat);
  cp.rhat_t = rhat_t;
  cp.goo = reinterpret_cast<float*>(ws + p->off_goo);
  cp.gjo = reinterpret_cast<float2*>(ws + p->off_gjo);
  cp.inv_G = (float)(1.0 / ((double)p->ny * (double)p->nx));
  cp.n_pair = p->n_pair;
  cp.scale = (float)(1.0 / ((double)(p->N - 1) * (double)p->ny * (double)p->nx));
  cp.vsel = p->sched[kPassStats];
  cp.twY = p->twY(cp.vsel);
  cp.status = p->d_status;
  if (wait_before_stats) {
    e = cudaStreamWaitEvent(s, wait_before_stats, 0);
    if (e != cudaSuccess) return e;
  }
  if (!rhat_t && p->use_fused()) {   // statistics only: the fused column pass writes the tables
    ColFusedParams f = fused_params(p, ws);
    f.chat = cp.chat;
    prof_begin(p, kPassFused, s);
    e = launch_col_fused(f, s);
    prof_end(p, kPassFused, s);
    return e;
  }
  prof_begin(p, kPassStats, s);
  e = launch_col_stats(cp, s);
  prof_end(p, kPassStats, s);
  return e;
}

extern "C" fftenkf_status fftenkf_estimate_spectrum(fftenkf_plan p, const void* ensemble, double* spectrum_out,
                                                    void* workspace, void* stream) {
  g_last_error.clear();
  if (!p || !ensemble || !spectrum_out) return fail(FFTENKF_EINVAL, "null argument");
  if (!aligned(ensemble, 16) || !aligned(spectrum_out, 16)) return fail(FFTENKF_EINVAL, "pointers must be 16-byte aligned");
  if (p->n_obs == 0) return FFTENKF_OK;   // no tables
  char* ws;
  fftenkf_status st = get_workspace(p, workspace, &ws);
  if (st != FFTENKF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = run_statistics(p, ensemble, ws, s, nullptr);
  prof_begin(p, kPassChatOut, s);
  if (e == cudaSuccess)
    e = launch_chat_out(reinterpret_cast<float*>(ws + p->off_chat), spectrum_out, p->ny, p->L,
                        chat_out_map(p->n_obs, p->n_un, p->coupled ? 1 : 0, p->obs, p->un, p->M), s);
  prof_end(p, kPassChatOut, s);
  if (e != cudaSuccess) return cuda_fail(e, "estimate_spectrum");
  return FFTENKF_OK;
}

// the analysis with given perturbations, or (drawn) with perturbations drawn in frequency space
static fftenkf_status analyze_impl(fftenkf_plan p, void* ensemble, const float* data, const void* perturbations,
                                   const double* rhat, const double* spectrum, bool drawn, unsigned long long seed,
                                   void* workspace, void* stream) {
  g_last_error.clear();
  if (!p || !ensemble) return fail(FFTENKF_EINVAL, "null argument");
  if (p->n_obs == 0) return FFTENKF_OK;   // nothing observed: the forecast is the analysis
  if (!data || (!perturbations && !drawn) || !rhat) return fail(FFTENKF_EINVAL, "null argument");
  if (!aligned(ensemble, 16) || !aligned(data, 16) || (!drawn && !aligned(perturbations, 16)) || !aligned(rhat, 16) ||
      (spectrum && !aligned(spectrum, 16)))
    return fail(FFTENKF_EINVAL, "pointers must be 16-byte aligned");
  if (spectrum && p->coupled)
    return fail(FFTENKF_EUNSUPPORTED, "a caller-supplied spectrum is not supported with coupled observed blocks");
  char* ws;
  fftenkf_status st = get_workspace(p, workspace, &ws);
  if (st != FFTENKF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  // auxiliary stream: rhat transposed for the gains (estimated spectrum) or the gain pass
  // (caller spectrum), overlapping the passes on the caller's stream
  e = cudaEventRecord(p->ev_fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->aux, p->ev_fork, 0);
  GainParams gp;
  memset(&gp, 0, sizeof(gp));
  gp.ny = p->ny; gp.L = p->L; gp.n_obs = p->n_obs; gp.n_un = p->n_un;
  gp.spec = spectrum;
  gp.rhat = rhat;
  gp.goo = reinterpret_cast<float*>(ws + p->off_goo);
  gp.gjo = reinterpret_cast<float2*>(ws + p->off_gjo);
  gp.scale = (float)(1.0 / ((double)p->ny * (double)p->nx));
  gp.status = p->d_status;
  double* rhat_t = reinterpret_cast<double*>(ws + p->off_rhat_t);
  if (spectrum && drawn) {   // the drawn perturbations scale by sqrt(rhat) in the column layout
    prof_begin(p, kPassRhatT, p->aux);
    if (e == cudaSuccess) e = launch_rhat_transpose(rhat, rhat_t, p->n_obs, p->ny, p->L, p->aux);
    prof_end(p, kPassRhatT, p->aux);
  }
  const bool fused = !spectrum && p->use_fused();
  float* amp_t = reinterpret_cast<float*>(ws + p->off_amp);
  if (!spectrum) {
    // the fused pass draws perturbations with the FP32 amplitudes sqrt(ny nx rhat) of the same pass
    prof_begin(p, kPassRhatT, p->aux);
    if (e == cudaSuccess)
      e = launch_rhat_transpose(rhat, rhat_t, p->n_obs, p->ny, p->L, p->aux, (fused && drawn) ? amp_t : nullptr,
                                (float)std::sqrt((double)p->ny * (double)p->nx));
    prof_end(p, kPassRhatT, p->aux);
  } else {
    prof_begin(p, kPassGain, p->aux);
    if (e == cudaSuccess) e = launch_gain(gp, p->aux);
    prof_end(p, kPassGain, p->aux);
  }
  if (e == cudaSuccess) e = cudaEventRecord(p->ev_join, p->aux);
  if (fused) {
    // anomaly rows now; the columns after the innovation rows
    if (e == cudaSuccess) e = run_anomaly_rows(p, ensemble, ws, s);
  } else if (!spectrum && p->coupled) {
    // tables of the column statistics, then the coupled gains (FP64 bracket inverse per wavenumber)
    if (e == cudaSuccess) e = run_statistics(p, ensemble, ws, s, nullptr);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_join, 0);
    CoupledGainParams cg;
    memset(&cg, 0, sizeof(cg));
    cg.ny = p->ny; cg.L = p->L; cg.n_obs = p->n_obs; cg.n_un = p->n_un; cg.n_pair = p->n_pair;
    cg.chat_t = reinterpret_cast<const float*>(ws + p->off_chat);
    cg.rhat_t = rhat_t;
    cg.gall = gp.gjo;
    cg.inv_G = (float)(1.0 / ((double)p->ny * (double)p->nx));
    cg.status = p->d_status;
    prof_begin(p, kPassGain, s);
    if (e == cudaSuccess) e = launch_coupled_gain(cg, s);
    prof_end(p, kPassGain, s);
  } else if (!spectrum) {
    // anomaly rows need no rhat; the statistics pass (which forms the gains) waits for it
    if (e == cudaSuccess) e = run_statistics(p, ensemble, ws, s, rhat_t, p->ev_join);
  } else {
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_join, 0);
  }
  RowFwdParams rp;
  memset(&rp, 0, sizeof(rp));
  rp.ny = p->ny; rp.nx = p->nx; rp.L = p->L; rp.M = p->M; rp.N = p->N;
  rp.n_obs = p->n_obs; rp.mode = drawn ? kInnovationDrawn : kInnovation; rp.storage = p->storage;
  for (int i = 0; i < p->n_obs; ++i) rp.obs[i] = p->obs[i];
  rp.ens = ensemble; rp.data = data; rp.pert = perturbations;
  rp.out = reinterpret_cast<float2*>(ws + p->off_W);
  rp.vsel = p->sched[kPassRowInnov];
  rp.twL = p->twL(rp.vsel & 1); rp.twX = p->twX(); rp.status = p->d_status;
  prof_begin(p, kPassRowInnov, s);
  if (e == cudaSuccess) e = launch_row_fwd(rp, p->N * p->n_obs, s);
  prof_end(p, kPassRowInnov, s);
  ColUpdParams up;
  memset(&up, 0, sizeof(up));
  up.ny = p->ny; up.L = p->L; up.M = p->M; up.N = p->N; up.n_obs = p->n_obs; up.n_un = p->n_un;
  for (int j = 0; j < p->M; ++j) {
    up.obs_of_block[j] = p->obs_of_block[j];
    up.un_of_block[j] = p->un_of_block[j];
  }
  up.W = rp.out; up.goo = gp.goo; up.gjo = gp.gjo;
  up.coupled = p->coupled ? 1 : 0;
  up.gall = gp.gjo;
  up.drawn = drawn ? 1 : 0;
  up.seed = seed;
  up.rhat_t = rhat_t;
  up.sqrt_G = (float)std::sqrt((double)p->ny * (double)p->nx);
  up.S = reinterpret_cast<float2*>(ws + p->off_A);
  up.vsel = p->sched[kPassUpdate];
  up.twY = p->twY(up.vsel); up.status = p->d_status;
  if (fused) {
    ColFusedParams f = fused_params(p, ws);
    f.W = rp.out;
    f.rhat_t = rhat_t;
    f.drawn = drawn ? 1 : 0;
    f.seed = seed;
    f.amp_t = amp_t;
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_join, 0);
    prof_begin(p, kPassFused, s);
    if (e == cudaSuccess) e = launch_col_fused(f, s);
    prof_end(p, kPassFused, s);
  } else {
    prof_begin(p, kPassUpdate, s);
    if (e == cudaSuccess) e = launch_col_update(up, s);
    prof_end(p, kPassUpdate, s);
  }
  RowInvParams ip;
  memset(&ip, 0, sizeof(ip));
  ip.ny = p->ny; ip.nx = p->nx; ip.L = p->L; ip.M = p->M; ip.N = p->N; ip.storage = p->storage;
  ip.vsel = p->sched[kPassRowInv];
  ip.ens = ensemble; ip.twL = p->twL(ip.vsel & 1); ip.twX = p->twX(); ip.status = p->d_status;
  ip.R = row_inv_rows(p->L, ip.vsel, p->ny, p->nx, p->storage == FFTENKF_BF16 ? 2 : 4);
  // columns per tensor copy: the largest divisor of L that is at most 256
  ip.box_cols = p->L < 256 ? p->L : 256;
  while (p->L % ip.box_cols) --ip.box_cols;
  if (p->tm_S != up.S || p->tm_R != ip.R) {   // re-encoded when the workspace or the item rows change
    p->tm_ok = encode_increment_map(&p->tm, up.S, p->M * p->N, p->ny, p->L, ip.R, ip.box_cols);
    p->tm_S = up.S;
    p->tm_R = ip.R;
  }
  if (!p->tm_ok && e == cudaSuccess) return fail(FFTENKF_ECUDA, "analyze: tensor map of the increment spectra refused");
  ip.tm_in = p->tm;
  prof_begin(p, kPassRowInv, s);
  if (e == cudaSuccess) e = launch_row_inv(ip, p->M * p->N, s);
  prof_end(p, kPassRowInv, s);
  if (e != cudaSuccess) return cuda_fail(e, "analyze");
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_analyze(fftenkf_plan p, void* ensemble, const float* data, const void* perturbations,
                                          const double* rhat, const double* spectrum, void* workspace, void* stream) {
  return analyze_impl(p, ensemble, data, perturbations, rhat, spectrum, false, 0, workspace, stream);
}

extern "C" fftenkf_status fftenkf_analyze_seeded(fftenkf_plan p, void* ensemble, const float* data, const double* rhat,
                                                 const double* spectrum, unsigned long long seed, void* workspace,
                                                 void* stream) {
  return analyze_impl(p, ensemble, data, nullptr, rhat, spectrum, true, seed, workspace, stream);
}

extern "C" fftenkf_status fftenkf_last_device_status(fftenkf_plan p, void* stream) {
  if (!p) return fail(FFTENKF_EINVAL, "null argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "stream");
  int word = 0;
  e = cudaMemcpy(&word, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "status word");
  if (word & kStatusTimeout) return fail(FFTENKF_ETIMEOUT, "a bounded wait for an asynchronous copy gave up");
  if (word & kStatusNonFinite) return fail(FFTENKF_ENONFINITE, "non-finite spectral covariance");
  return FFTENKF_OK;
}

extern "C" const char* fftenkf_status_string(fftenkf_status s) {
  switch (s) {
    case FFTENKF_OK: return "ok";
    case FFTENKF_EINVAL: return "invalid argument";
    case FFTENKF_EUNSUPPORTED: return "unsupported size or configuration";
    case FFTENKF_ECUDA: return "CUDA error";
    case FFTENKF_ENONFINITE: return "non-finite spectral covariance";
    case FFTENKF_ETIMEOUT: return "device wait timed out";
    case FFTENKF_ENOMEM: return "out of device memory";
  }
  return "unknown status";
}

extern "C" const char* fftenkf_last_error(void) { return g_last_error.c_str(); }

extern "C" fftenkf_status fftenkf_set_profiling(fftenkf_plan p, int enable) {
  if (!p) return fail(FFTENKF_EINVAL, "null argument");
  p->prof = enable != 0;
  for (int a = 0; a < kPassCount; ++a) {
    p->used[a] = 0;
    p->acc_ms[a] = 0.0;
    p->launches[a] = 0;
  }
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_pass_times(fftenkf_plan p, double* total_ms, int* launches, int n_passes) {
  if (!p || !total_ms || !launches) return fail(FFTENKF_EINVAL, "null argument");
  for (int a = 0; a < kPassCount; ++a) {
    const int n = p->used[a] < fftenkf_plan_s::kSlots ? p->used[a] : fftenkf_plan_s::kSlots;
    const int first = p->used[a] < fftenkf_plan_s::kSlots ? 0 : p->used[a] % fftenkf_plan_s::kSlots;
    for (int i = 0; i < n; ++i) prof_drain(p, a, (first + i) % fftenkf_plan_s::kSlots);
    if (a < n_passes) {
      total_ms[a] = p->acc_ms[a];
      launches[a] = p->launches[a];
    }
    p->used[a] = 0;
    p->acc_ms[a] = 0.0;
    p->launches[a] = 0;
  }
  return FFTENKF_OK;
}

extern "C" int fftenkf_pass_count(void) { return kPassCount; }

extern "C" const char* fftenkf_pass_name(int pass) {
  return (pass >= 0 && pass < kPassCount) ? kPassNames[pass] : "";
}

extern "C" fftenkf_status fftenkf_set_schedule(fftenkf_plan p, const int* sched, int n) {
  if (!p || !sched || n < 0) return fail(FFTENKF_EINVAL, "null argument");
  const int nf = table_floats(p);
  int next[kPassCount];
  for (int a = 0; a < kPassCount; ++a) next[a] = (a < n) ? sched[a] : p->sched[a];
  for (int a = 0; a < kPassCount; ++a) {
    const bool row_pass = (a == kPassRowAnom || a == kPassRowInnov || a == kPassRowInv);
    if (next[a] < 0 || next[a] > (row_pass ? 3 : 1)) return fail(FFTENKF_EINVAL, "schedule entry out of range");
  }
  if (p->n_obs > 0 && (col_stats_smem(p->ny, nf, next[kPassStats], nullptr) == 0 ||
                       col_update_smem(p->ny, p->n_obs, next[kPassUpdate], nullptr, nullptr) == 0 ||
                       row_inv_rows(p->L, next[kPassRowInv], p->ny, p->nx, p->storage == FFTENKF_BF16 ? 2 : 4) == 0))
    return fail(FFTENKF_EUNSUPPORTED, "schedule does not fit in shared memory");
  for (int a = 0; a < kPassCount; ++a) p->sched[a] = next[a];
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_set_coupled(fftenkf_plan p, int coupled) {
  g_last_error.clear();
  if (!p) return fail(FFTENKF_EINVAL, "null argument");
  const bool c = coupled != 0;
  if (c && (p->n_obs < 1 || p->n_obs > 2))
    return fail(FFTENKF_EUNSUPPORTED, "coupled observed blocks: one or two observed blocks supported");
  const int n_pair = c ? p->n_obs * (p->n_obs - 1) / 2 : 0;
  const int nf = p->n_obs + 2 * n_pair + 2 * p->n_obs * p->n_un;
  if (p->n_obs > 0 && col_stats_smem(p->ny, nf, p->sched[kPassStats], nullptr) == 0)
    return fail(FFTENKF_EUNSUPPORTED, "coupled covariance tables per column exceed shared memory (reduce blocks or ny)");
  if (c == p->coupled) return FFTENKF_OK;
  p->coupled = c;
  p->n_pair = n_pair;
  const size_t old_bytes = p->ws_bytes;
  layout(p);
  if (p->own_ws && p->ws_bytes > old_bytes) {   // reallocated on the next call
    cudaFree(p->own_ws);
    p->own_ws = nullptr;
  }
  p->tm_S = nullptr;   // the tensor map is encoded again for the new layout
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_set_expire_first_wait(fftenkf_plan p, int on) {
  if (!p) return fail(FFTENKF_EINVAL, "null argument");
  p->expire_first_wait = on ? 1 : 0;
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_get_schedule(fftenkf_plan p, int* sched, int n) {
  if (!p || !sched) return fail(FFTENKF_EINVAL, "null argument");
  for (int a = 0; a < kPassCount && a < n; ++a) sched[a] = p->sched[a];
  return FFTENKF_OK;
}
