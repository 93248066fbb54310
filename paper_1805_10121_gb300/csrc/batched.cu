// Grouped Chebyshev filter over many independent problems (Alg. 4 applied to
// a batch of Hermitian matrices of different sizes).
//
// The paper filters one matrix at a time; a batch of small problems (N of a
// few hundred to a few thousand) leaves most of GB300's 152 SMs idle when
// each product is its own launch.  Here every degree step of the filter is
// one launch over the output tiles of all problems that still have active
// columns: CTA t finds its problem by binary search over the step's tile
// prefix, so the hardware block scheduler hands the next tile of any problem
// to whichever SM frees up (problems are ordered by decreasing N, longest
// tiles first).  Per problem the columns are sorted by degree (Alg. 4 lines
// 12-14 keep an active suffix), the recurrence coefficients of Eq. 7 are
// computed on the host once per call, and the whole sequence of step
// launches is captured into a CUDA graph and launched once.
//
// FP64 products run on the DMMA kernel with one of four tile shapes chosen
// by timing the first step (which only writes the second buffer, so it can
// be repeated); the choice is cached per batch shape.  Split-BF16 products
// slice the active columns of every problem in one launch per step and run
// the tensor-core kernel with its fixed 128 x 32 complex tile.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

#include "chase.h"
#include "common.cuh"
#include "context.hpp"

namespace chase {
namespace {

constexpr int kMaxDegree = 1024;

// Per-problem constants of Alg. 4 lines 2-3 and the problem's place in the
// grouped order.
struct Coef {
  int q;  // index into the caller's input list
  double c, e, sigma1;
};

// Step list of degree step i (1-based) for a tile shape bm x bn, where bn
// counts B-map columns (complex columns for FP64, real ones for split);
// real_cols = 2 for split, 1 for FP64.  sigma_prev[k] is sigma after step
// i - 1 of problem k (Alg. 4 line 11).
void build_step(const std::vector<GroupedFilterInput>& in, const std::vector<Coef>& co, int i,
                int bm, int bn, int real_cols, const std::vector<double>& sigma_prev,
                std::vector<GroupedStep>& out, int* ntiles, int* ncols) {
  out.clear();
  int tiles = 0, cols = 0;
  for (size_t k = 0; k < co.size(); ++k) {
    const GroupedFilterInput& pi = in[co[k].q];
    if (i > pi.maxdeg) continue;
    const int s = pi.start[i];
    if (s >= pi.b) continue;
    GroupedStep g;
    g.prob = static_cast<int>(k);
    g.s = s;
    g.tile0 = tiles;
    g.col0 = cols;
    if (i == 1) {  // Alg. 4 line 4
      g.alpha = co[k].sigma1 / co[k].e;
      g.beta = 0.0;
    } else {  // lines 8-9
      const double sigma = sigma_prev[k];
      const double tau = 1.0 / (2.0 / co[k].sigma1 - sigma);
      g.alpha = 2.0 * tau / co[k].e;
      g.beta = -tau * sigma;
    }
    g.shift = co[k].c;
    out.push_back(g);
    const int rt = (pi.n + bm - 1) / bm;
    const int ct = (real_cols * (pi.b - s) + bn - 1) / bn;
    tiles += rt * ct;
    cols += pi.b - s;
  }
  GroupedStep sentinel{};
  sentinel.prob = -1;
  sentinel.tile0 = tiles;
  sentinel.col0 = cols;
  out.push_back(sentinel);
  *ntiles = tiles;
  *ncols = cols;
}

std::mutex g_tune_mu;
std::map<std::tuple<int, long long, long long, int, int>, int> g_tune_cache;

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct GraphGuard {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  cudaStream_t cs = nullptr;
  ~GraphGuard() {
    if (x) cudaGraphExecDestroy(x);
    if (g) cudaGraphDestroy(g);
    if (cs) cudaStreamDestroy(cs);
  }
};

struct EventPool {
  std::vector<cudaEvent_t> ev;
  cudaEvent_t get() {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    ev.push_back(e);
    return e;
  }
  ~EventPool() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

float elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return 0.f;
  return ms;
}

}  // namespace

int grouped_split_prepare(Dev& d, std::vector<GroupedFilterInput>& in, const std::vector<int>& bcap) {
  std::vector<GroupedSliceH> hs;
  int rows = 0;
  for (size_t q = 0; q < in.size(); ++q) {
    GroupedFilterInput& g = in[q];
    if (g.n == 0) continue;
    const int64_t Kp = split_k_padded(g.n);
    CHASE_TRY(d.alloc_bytes(&g.A, static_cast<size_t>(kSplitSlices) * g.n * Kp * 2));
    CHASE_TRY(d.alloc(&g.E, static_cast<size_t>(g.n)));
    CHASE_TRY(d.alloc(&g.Dg, static_cast<size_t>(g.n)));
    g.bcap = std::max(bcap[q], 1);
    CHASE_TRY(d.alloc_bytes(&g.Bsl, static_cast<size_t>(kSplitSlices) * 2 * g.bcap * Kp * 2));
    CHASE_TRY(d.alloc(&g.F, static_cast<size_t>(g.bcap)));
    GroupedSliceH sh;
    sh.H = reinterpret_cast<const double2*>(g.H);
    sh.ldh = g.ldh;
    sh.A = g.A;
    sh.E = g.E;
    sh.Dg = g.Dg;
    sh.Kp = Kp;
    sh.n = g.n;
    sh.row0 = rows;
    hs.push_back(sh);
    rows += g.n;
  }
  if (hs.empty()) return CHASE_OK;
  GroupedSliceH* dsl = nullptr;
  CHASE_TRY(d.alloc(&dsl, hs.size()));
  CHASE_CUDA(cudaMemcpyAsync(dsl, hs.data(), sizeof(GroupedSliceH) * hs.size(),
                             cudaMemcpyHostToDevice, d.st));
  CHASE_TRY(split_grouped_prepare_h(d, dsl, static_cast<int>(hs.size()), rows));
  // the host array must outlive the copy
  return d.sync_check("grouped slices of H");
}

int grouped_filter_sorted(Dev& d, const std::vector<GroupedFilterInput>& in, bool split, int tile,
                          GroupedFilterTimes* times) {
  const long long launches0 = chase_kernel_launches();
  GroupedFilterTimes tt;
  // active problems, longest tiles first: the block scheduler then balances the tail
  std::vector<Coef> co;
  int maxdeg = 0;
  for (size_t q = 0; q < in.size(); ++q) {
    const GroupedFilterInput& g = in[q];
    if (g.n == 0 || g.b == 0) continue;
    Coef c;
    c.q = static_cast<int>(q);
    c.c = 0.5 * (g.b_sup + g.mu_nn);  // Alg. 4 line 2
    c.e = 0.5 * (g.b_sup - g.mu_nn);
    c.sigma1 = c.e / (g.mu1 - c.c);   // line 3
    co.push_back(c);
    maxdeg = std::max(maxdeg, g.maxdeg);
  }
  std::stable_sort(co.begin(), co.end(),
                   [&](const Coef& x, const Coef& y) { return in[x.q].n > in[y.q].n; });
  const int Q = static_cast<int>(co.size());
  if (Q == 0) {
    if (times) *times = tt;
    return CHASE_OK;
  }
  EventPool evp;
  const int nmaps = split ? 2 : 3;
  CUtensorMap* dmaps = nullptr;
  CHASE_TRY(d.alloc_bytes(reinterpret_cast<void**>(&dmaps), sizeof(CUtensorMap) * nmaps * Q));
  GroupedProblem* dprobs = nullptr;
  CHASE_TRY(d.alloc(&dprobs, Q));
  std::vector<GroupedProblem> probs(Q);
  std::vector<CUtensorMap> maps(static_cast<size_t>(nmaps) * Q);
  for (int k = 0; k < Q; ++k) {
    const GroupedFilterInput& pi = in[co[k].q];
    GroupedProblem& g = probs[k];
    g = GroupedProblem{};
    g.n = pi.n;
    g.b = pi.b;
    g.buf0 = reinterpret_cast<double2*>(pi.X);
    g.ld0 = pi.ldx;
    g.buf1 = reinterpret_cast<double2*>(pi.W);
    g.ld1 = pi.ldw;
    g.mapA = dmaps + nmaps * k;
    g.mapB0 = dmaps + nmaps * k + 1;
    g.mapB1 = split ? nullptr : dmaps + nmaps * k + 2;
    if (split) {
      if (!pi.A || !pi.Bsl || pi.bcap < pi.b) {
        set_error("grouped filter: slice workspace missing or too small");
        return CHASE_INVALID_ARG;
      }
      const int64_t Kp = split_k_padded(pi.n);
      g.Kp = Kp;
      g.E = pi.E;
      g.F = pi.F;
      g.Dg = pi.Dg;
      g.Bsl = pi.Bsl;
      g.bcap = pi.bcap;
      CHASE_TRY(make_tmap_bf16_3d(&maps[nmaps * k], pi.A, 2LL * pi.n, pi.n, kSplitSlices, Kp * 2,
                                  Kp * 2 * pi.n, kSplitStageK, kSplitTileRows, kSplitSlices));
      CHASE_TRY(make_tmap_bf16_3d(&maps[nmaps * k + 1], pi.Bsl, 2LL * pi.n, 2LL * pi.b, kSplitSlices,
                                  Kp * 2, Kp * 2 * 2 * pi.bcap, kSplitStageK, kSplitTileRealCols,
                                  kSplitSlices));
    }
  }
  CHASE_CUDA(cudaMemcpyAsync(dprobs, probs.data(), sizeof(GroupedProblem) * Q, cudaMemcpyHostToDevice,
                             d.st));
  // FP64 maps depend on the tile shape: encoded after the tile choice.
  auto encode_fp64_maps = [&](int cfg) -> int {
    int bm = 0, bn = 0;
    grouped_fp64_tile(cfg, &bm, &bn);
    for (int k = 0; k < Q; ++k) {
      const GroupedFilterInput& pi = in[co[k].q];
      CHASE_TRY(make_tmap_c64(&maps[nmaps * k], pi.H, pi.n, pi.n, pi.ldh, bm, 16));
      CHASE_TRY(make_tmap_c64(&maps[nmaps * k + 1], pi.X, pi.n, pi.b, pi.ldx, 16, bn));
      CHASE_TRY(make_tmap_c64(&maps[nmaps * k + 2], pi.W, pi.n, pi.b, pi.ldw, 16, bn));
    }
    CHASE_CUDA(cudaMemcpyAsync(dmaps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                               cudaMemcpyHostToDevice, d.st));
    // the host array is rewritten by the next encoding: finish this copy first
    CHASE_CUDA(cudaStreamSynchronize(d.st));
    return CHASE_OK;
  };

  int cfg = -1;
  if (split) {
    CHASE_CUDA(cudaMemcpyAsync(dmaps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                               cudaMemcpyHostToDevice, d.st));
  } else if (tile != CHASE_TILE_AUTO) {
    cfg = tile;
  } else {
    long long sum_n = 0, sum_nb = 0;
    int max_n = 0;
    for (const Coef& c : co) {
      sum_n += in[c.q].n;
      sum_nb += static_cast<long long>(in[c.q].n) * in[c.q].b;
      max_n = std::max(max_n, in[c.q].n);
    }
    const auto key = std::make_tuple(Q, sum_n, sum_nb, max_n, maxdeg);
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) cfg = it->second;
    }
    if (cfg < 0) {
      // time step 1 (reads X, writes W only) with every tile shape
      const double ta = now_s();
      float best = 0.f;
      std::vector<double> sigma0(Q, 0.0);
      for (int c = 0; c < kGroupedFp64Cfgs; ++c) {
        int bm = 0, bn = 0;
        grouped_fp64_tile(c, &bm, &bn);
        std::vector<GroupedStep> one;
        int nt = 0, nc = 0;
        build_step(in, co, 1, bm, bn, 1, sigma0, one, &nt, &nc);
        GroupedStep* dst1 = nullptr;
        CHASE_TRY(d.alloc(&dst1, one.size()));
        CHASE_CUDA(cudaMemcpyAsync(dst1, one.data(), sizeof(GroupedStep) * one.size(),
                                   cudaMemcpyHostToDevice, d.st));
        CHASE_TRY(encode_fp64_maps(c));
        cudaEvent_t ea = evp.get(), eb = evp.get();
        if (!ea || !eb) {
          set_error("grouped filter: event creation failed");
          return CHASE_CUDA_ERROR;
        }
        const int na = static_cast<int>(one.size()) - 1;
        // one untimed launch, then the timed one
        CHASE_TRY(zgemm_grouped_fp64(d, c, dprobs, dst1, na, nt, 0));
        CHASE_CUDA(cudaEventRecord(ea, d.st));
        CHASE_TRY(zgemm_grouped_fp64(d, c, dprobs, dst1, na, nt, 0));
        CHASE_CUDA(cudaEventRecord(eb, d.st));
        CHASE_TRY(d.sync_check("grouped filter autotune"));
        const float ms = elapsed_ms(ea, eb);
        if (cfg < 0 || ms < best) {
          best = ms;
          cfg = c;
        }
      }
      tt.t_autotune = now_s() - ta;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[key] = cfg;
    }
  }
  int bm = kSplitTileRows, bn = kSplitTileRealCols, realc = 2;
  if (!split) {
    grouped_fp64_tile(cfg, &bm, &bn);
    realc = 1;
    CHASE_TRY(encode_fp64_maps(cfg));
  }
  // ---- every step's list, uploaded once ----
  std::vector<GroupedStep> all, one;
  std::vector<int> first(maxdeg + 1, 0), nact(maxdeg + 1, 0), ntiles(maxdeg + 1, 0),
      ncols(maxdeg + 1, 0);
  {
    std::vector<double> sigma(Q, 0.0);
    for (int i = 1; i <= maxdeg; ++i) {
      build_step(in, co, i, bm, bn, realc, sigma, one, &ntiles[i], &ncols[i]);
      first[i] = static_cast<int>(all.size());
      nact[i] = static_cast<int>(one.size()) - 1;
      all.insert(all.end(), one.begin(), one.end());
      for (int k = 0; k < Q; ++k) {  // Alg. 4 line 11
        if (i == 1)
          sigma[k] = co[k].sigma1;
        else if (i <= in[co[k].q].maxdeg)
          sigma[k] = 1.0 / (2.0 / co[k].sigma1 - sigma[k]);
      }
    }
  }
  GroupedStep* dsteps = nullptr;
  CHASE_TRY(d.alloc(&dsteps, all.size()));
  CHASE_CUDA(cudaMemcpyAsync(dsteps, all.data(), sizeof(GroupedStep) * all.size(),
                             cudaMemcpyHostToDevice, d.st));

  // ---- the degree steps, captured into one graph ----
  CHASE_TRY(split ? zgemm_split_grouped_prepare() : zgemm_grouped_fp64_prepare(cfg));
  const double tg = now_s();
  GraphGuard gg;
  CHASE_CUDA(cudaStreamCreateWithFlags(&gg.cs, cudaStreamNonBlocking));
  std::vector<cudaEvent_t> pev;  // product start / end per step, inside the graph
  for (int i = 1; i <= maxdeg; ++i) {
    if (ntiles[i] == 0) continue;
    cudaEvent_t a = evp.get(), z = evp.get();
    if (!a || !z) {
      set_error("grouped filter: event creation failed");
      return CHASE_CUDA_ERROR;
    }
    pev.push_back(a);
    pev.push_back(z);
  }
  cudaEvent_t g_begin = evp.get(), g_end = evp.get();
  if (!g_begin || !g_end) {
    set_error("grouped filter: event creation failed");
    return CHASE_CUDA_ERROR;
  }
  {
    cudaStream_t user = d.st;
    d.st = gg.cs;
    int st = CHASE_OK;
    if (cudaStreamBeginCapture(gg.cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      d.st = user;
      set_error("grouped filter: stream capture failed to start");
      return CHASE_CUDA_ERROR;
    }
    size_t k = 0;
    for (int i = 1; i <= maxdeg && st == CHASE_OK; ++i) {
      if (ntiles[i] == 0) continue;
      const int parity = (i - 1) & 1;
      const GroupedStep* sp = dsteps + first[i];
      if (split) st = split_grouped_slice_x(d, dprobs, sp, nact[i], ncols[i], parity);
      if (st != CHASE_OK) break;
      // external records: real event nodes of the graph, so the product
      // launches can be timed apart from the slicing
      if (cudaEventRecordWithFlags(pev[k], gg.cs, cudaEventRecordExternal) != cudaSuccess)
        st = CHASE_CUDA_ERROR;
      if (st == CHASE_OK)
        st = split ? zgemm_split_grouped(d, dprobs, sp, nact[i], ntiles[i], parity)
                   : zgemm_grouped_fp64(d, cfg, dprobs, sp, nact[i], ntiles[i], parity);
      if (st == CHASE_OK &&
          cudaEventRecordWithFlags(pev[k + 1], gg.cs, cudaEventRecordExternal) != cudaSuccess)
        st = CHASE_CUDA_ERROR;
      k += 2;
    }
    const cudaError_t ec = cudaStreamEndCapture(gg.cs, &gg.g);
    d.st = user;
    if (st != CHASE_OK) return st;
    if (ec != cudaSuccess || !gg.g) {
      set_error("grouped filter: stream capture failed: %s", cudaGetErrorString(ec));
      return CHASE_CUDA_ERROR;
    }
  }
  CHASE_CUDA(cudaGraphInstantiate(&gg.x, gg.g, 0));
  tt.t_graph_build = now_s() - tg;
  CHASE_CUDA(cudaEventRecord(g_begin, d.st));
  CHASE_CUDA(cudaGraphLaunch(gg.x, d.st));
  CHASE_CUDA(cudaEventRecord(g_end, d.st));
  CHASE_TRY(d.sync_check("grouped filter"));
  // With even degrees the last product of every column lands in X.
  for (const Coef& c : co) {
    const GroupedFilterInput& pi = in[c.q];
    for (int i = 1; i <= pi.maxdeg; ++i) {
      const int a = pi.b - pi.start[i];
      tt.matvecs += a;
      tt.flops += 8.0 * pi.n * static_cast<double>(pi.n) * a;
    }
  }
  for (size_t k = 0; k < pev.size(); k += 2) tt.t_product += 1e-3 * elapsed_ms(pev[k], pev[k + 1]);
  tt.t_steps = 1e-3 * elapsed_ms(g_begin, g_end);
  cudaGetLastError();  // a timing query that failed leaves no error behind
  tt.tile_config = cfg;
  tt.steps = maxdeg;
  tt.launches = static_cast<int>(chase_kernel_launches() - launches0);
  if (times) *times = tt;
  return CHASE_OK;
}

}  // namespace chase

using namespace chase;

extern "C" int chase_filter_batched(int P, const chase_c64* const* H, const int64_t* N,
                                    const int64_t* ldh, chase_c64* const* V, const int64_t* ldv,
                                    const int* b, const int* const* degrees, const double* b_sup,
                                    const double* mu1, const double* mu_nevnex, int precision,
                                    int tile, chase_batch_stats* stats, void* stream) {
  const double t0 = now_s();
  const long long launches0 = chase_kernel_launches();
  if (stats) *stats = chase_batch_stats{};
  if (precision != CHASE_FP64 && precision != CHASE_SPLIT_BF16) {
    set_error("chase_filter_batched: unknown precision %d", precision);
    return CHASE_INVALID_ARG;
  }
  if (tile < CHASE_TILE_AUTO || tile >= kGroupedFp64Cfgs) {
    set_error("chase_filter_batched: tile must be CHASE_TILE_AUTO or 0..%d", kGroupedFp64Cfgs - 1);
    return CHASE_INVALID_ARG;
  }
  if (P < 0 || (P > 0 && (!H || !N || !ldh || !V || !ldv || !b || !degrees || !b_sup || !mu1 ||
                          !mu_nevnex))) {
    set_error("chase_filter_batched: invalid problem count or NULL array");
    return CHASE_INVALID_ARG;
  }
  // ---- validation and the column order of every problem ----
  std::vector<int> idx;                    // caller's index of each problem with work
  std::vector<std::vector<int>> perm, start;
  for (int p = 0; p < P; ++p) {
    const int64_t n = N[p];
    if (n < 0 || b[p] < 0 || n > (1 << 20) || ldh[p] < std::max<int64_t>(1, n) ||
        ldv[p] < std::max<int64_t>(1, n)) {
      set_error("chase_filter_batched: problem %d: invalid size or leading dimension", p);
      return CHASE_INVALID_ARG;
    }
    if (n == 0 || b[p] == 0) continue;
    if (!H[p] || !V[p] || !degrees[p]) {
      set_error("chase_filter_batched: problem %d: NULL array", p);
      return CHASE_INVALID_ARG;
    }
    if (!is_device_ptr(H[p]) || !is_device_ptr(V[p])) {
      set_error("chase_filter_batched: problem %d: H and V must be device arrays", p);
      return CHASE_INVALID_ARG;
    }
    if (!(mu1[p] < mu_nevnex[p] && mu_nevnex[p] < b_sup[p]) || !std::isfinite(b_sup[p]) ||
        !std::isfinite(mu1[p])) {
      set_error("chase_filter_batched: problem %d: need mu1 < mu_nevnex < b_sup", p);
      return CHASE_INVALID_ARG;
    }
    const int* deg = degrees[p];
    int mx = 0;
    for (int j = 0; j < b[p]; ++j) {
      const int m = deg[j];
      if (m < 2 || m > kMaxDegree || (m & 1)) {
        set_error("chase_filter_batched: problem %d column %d: degree %d not even in [2, %d]", p, j,
                  m, kMaxDegree);
        return CHASE_INVALID_ARG;
      }
      mx = std::max(mx, m);
    }
    std::vector<int> pm(b[p]);
    std::iota(pm.begin(), pm.end(), 0);
    std::stable_sort(pm.begin(), pm.end(), [&](int x, int y) { return deg[x] < deg[y]; });
    std::vector<int> st(mx + 2, 0);  // Alg. 4 lines 12-14: columns of degree < i
    int s = 0;
    for (int i = 0; i <= mx + 1; ++i) {
      while (s < b[p] && deg[pm[s]] < i) ++s;
      st[i] = s;
    }
    idx.push_back(p);
    perm.push_back(std::move(pm));
    start.push_back(std::move(st));
  }
  const int Q = static_cast<int>(idx.size());
  if (Q == 0) return CHASE_OK;
  const bool split = precision == CHASE_SPLIT_BF16;

  Dev d(stream);
  CHASE_TRY(d.init());
  // sorted copies of the blocks (the filter's X), V is the second buffer
  std::vector<size_t> off0(Q);
  size_t tot0 = 0, totperm = 0;
  for (int q = 0; q < Q; ++q) {
    off0[q] = tot0;
    tot0 += (static_cast<size_t>(N[idx[q]]) * b[idx[q]] + 15) / 16 * 16;  // 256-byte aligned
    totperm += b[idx[q]];
  }
  chase_c64* buf0 = nullptr;
  int* dperm = nullptr;
  GroupedPermute* dgather = nullptr;
  GroupedPermute* dscatter = nullptr;
  CHASE_TRY(d.alloc(&buf0, tot0));
  CHASE_TRY(d.alloc(&dperm, totperm));
  CHASE_TRY(d.alloc(&dgather, Q));
  CHASE_TRY(d.alloc(&dscatter, Q));
  std::vector<int> hperm;
  hperm.reserve(totperm);
  std::vector<GroupedPermute> gat(Q), sca(Q);
  std::vector<GroupedFilterInput> in(Q);
  std::vector<int> bcap(Q);
  int total_cols = 0;
  for (int q = 0; q < Q; ++q) {
    const int p = idx[q];
    GroupedPermute& g = gat[q];
    g.src = reinterpret_cast<const double2*>(V[p]);
    g.lds = ldv[p];
    g.dst = reinterpret_cast<double2*>(buf0 + off0[q]);
    g.ldd = N[p];
    g.perm = dperm + hperm.size();
    g.n = static_cast<int>(N[p]);
    g.col0 = total_cols;
    GroupedPermute& h = sca[q];
    h = g;
    h.src = g.dst;
    h.lds = g.ldd;
    h.dst = reinterpret_cast<double2*>(V[p]);
    h.ldd = ldv[p];
    total_cols += b[p];
    hperm.insert(hperm.end(), perm[q].begin(), perm[q].end());
    GroupedFilterInput& f = in[q];
    f.H = H[p];
    f.ldh = ldh[p];
    f.n = static_cast<int>(N[p]);
    f.X = buf0 + off0[q];
    f.ldx = N[p];
    f.W = V[p];
    f.ldw = ldv[p];
    f.b = b[p];
    f.start = start[q].data();
    f.maxdeg = static_cast<int>(start[q].size()) - 2;
    f.b_sup = b_sup[p];
    f.mu1 = mu1[p];
    f.mu_nn = mu_nevnex[p];
    bcap[q] = b[p];
  }
  CHASE_CUDA(cudaMemcpyAsync(dperm, hperm.data(), sizeof(int) * hperm.size(), cudaMemcpyHostToDevice,
                             d.st));
  CHASE_CUDA(cudaMemcpyAsync(dgather, gat.data(), sizeof(GroupedPermute) * Q, cudaMemcpyHostToDevice,
                             d.st));
  CHASE_CUDA(cudaMemcpyAsync(dscatter, sca.data(), sizeof(GroupedPermute) * Q,
                             cudaMemcpyHostToDevice, d.st));
  CHASE_TRY(launch_grouped_permute(d, dgather, Q, total_cols, false));
  if (split) CHASE_TRY(grouped_split_prepare(d, in, bcap));
  GroupedFilterTimes tt;
  CHASE_TRY(grouped_filter_sorted(d, in, split, tile, &tt));
  // every result is in the sorted copy (even degrees): back to the caller's order
  CHASE_TRY(launch_grouped_permute(d, dscatter, Q, total_cols, true));
  CHASE_TRY(d.sync_check("chase_filter_batched"));
  if (stats) {
    stats->problems = Q;
    stats->steps = tt.steps;
    stats->tile_config = tt.tile_config;
    stats->launches = static_cast<int>(chase_kernel_launches() - launches0);
    stats->matvecs = tt.matvecs;
    stats->flops = tt.flops;
    stats->t_autotune = tt.t_autotune;
    stats->t_graph_build = tt.t_graph_build;
    stats->t_steps = tt.t_steps;
    stats->t_product = tt.t_product;
    stats->t_total = now_s() - t0;
  }
  return CHASE_OK;
}
