// Host side of the C ABI declared in include/pentbatch.h: plans, workspace
// layout, argument checks, dispatch and CUDA-graph time stepping.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <numeric>
#include <tuple>
#include <vector>

#include <cuda.h>  // CUpointer_attribute / CUmemorytype; the driver function comes through the runtime
#include <nvtx3/nvToolsExt.h>

#include "../../include/pentbatch.h"
#include "internal.cuh"

using namespace pent;

namespace {
// An NVTX range over one library call (header-only NVTX 3: free when no profiler is attached;
// host-side only, so it is allowed inside a stream capture).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};
}  // namespace

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Region {
  size_t off = 0, bytes = 0;
};

}  // namespace

struct pent_plan {
  // shapes
  int64_t batch = 0;
  std::vector<int64_t> n;    // rows per system
  std::vector<int64_t> off;  // batch + 1 offsets, caller layout
  int64_t rows = 0;
  bool uniform = true;
  int64_t n_uniform = 0;
  bool shared = false;
  pent_precision precision = PENT_F64;
  // options
  int threads_per_system = 1;
  int residual = PENT_RESIDUAL_FF;
  int block_warps = 2;
  int unroll = 4;
  int tol_log2 = 43;
  // tuning: rules from the tune cache, option overrides, FP64 launch runs
  struct Rule {
    int prec;
    int64_t lo, hi;
    int a, b;  // f32: rows per thread, threads per system; f64: unroll, block warps
  };
  std::vector<Rule> rules;
  int64_t rpt_override = 0;   // PENT_OPT_ROWS_PER_THREAD (0: not set)
  bool f64_explicit = false;  // PENT_OPT_UNROLL / PENT_OPT_BLOCK_WARPS set: one launch for all groups
  struct F64Run {
    int64_t g0, g1;  // groups [g0, g1)
    int unroll, bw;
    bool part;       // partitioned solve of long groups (chunks [c0, c1))
    int64_t c0, c1;
  };
  std::vector<F64Run> runs;
  // windowed walks of groups of long hyperdiffusion systems (csrc/core64.cu): windows of
  // win64_rows rows, one warp each, built at factor time from each group's overlap
  int win64_rows = 1024;          // PENT_OPT_WINDOW_ROWS (0: off)
  int win64_omax = 0;             // largest overlap a window takes (window rows / 8; / 4 for system windows)
  int64_t win64_cap = 0;          // windows the workspace holds
  int64_t nwin64 = 0;             // windows of the current factorisation (0: none)
  bool persistent = false;        // PENT_OPT_PERSISTENT: window launches as resident grids
  bool f64_interior = true;       // PENT_OPT_FP64_INTERIOR: hyperdiffusion walks take interior records from registers
  bool interior_valid = false;    // the interior records are those of the current factorisation
  // PENT_OPT_WINDOW_FORM 1: system windows (one thread per window of one system, the system's
  // own overlap, records copied per system at factor time); 0: group windows (one warp each)
  int win64_form = 1;
  int64_t swin_cap = 0;           // system windows the workspace holds
  int64_t srec_pairs = 0;         // row pairs of per-system records the workspace holds
  int64_t srec_maxpairs = 0;      // row pairs of the longest system that can take system windows
  std::vector<F64Run> wruns;      // the runs of the other groups
  int64_t part_rows = -1;  // PENT_OPT_PARTITION_ROWS (-1: automatic)
  bool periodic = false;   // PENT_OPT_PERIODIC: cyclic systems (Navon's reduction)
  // partitioned groups: chunk list and per-group chunk ranges
  std::vector<int32_t> pck, pcc, pcnum;
  std::vector<int64_t> pcbase;
  int64_t pchunks = 0;
  int64_t cfg_version = 0;  // bumped whenever launch settings change (graph cache key)
  // thread-per-system grouping (systems sorted by length, longest first)
  std::vector<int32_t> perm;  // [ngroups*32], -1 for padding lanes
  int64_t ngroups = 0;
  std::vector<int64_t> goff;
  std::vector<int32_t> glen;
  std::vector<int64_t> gmax;  // longest system of each group (unpadded)
  int64_t grows = 0;  // record rows over all groups
  // FP32 (refined) solve: per factored system a CTA shape (L rows per thread,
  // W warps per CTA, C CTAs per cluster), grouped into buckets of equal shape
  struct Shape {
    int L, W, C;
    bool operator<(const Shape& o) const { return std::tie(L, W, C) < std::tie(o.L, o.W, o.C); }
  };
  std::vector<Shape> shape;       // [nfac]
  std::vector<int64_t> foff;      // [nfac] float4 offset of each factor block
  int64_t fac_float4 = 0;         // total float4 of factor storage
  std::vector<int32_t> sys32;     // [batch] systems in bucket order
  std::vector<F32Bucket> buckets;
  int64_t tps_override = 0;       // PENT_OPT_THREADS_PER_SYSTEM for FP32 (0: automatic)
  int cluster_warps = 8;          // PENT_OPT_CLUSTER_WARPS
  int f32_kernel = 0;             // PENT_OPT_FP32_KERNEL: 0 interior-constant kernel where it applies, 1 general
  // windowed solve of long systems (csrc/f32u.cu): CTAs of win_warps warps, 8 rows a thread, each
  // solving one window of a system longer than one CTA; built at factor time from each system's
  // overlap (k_uplan32)
  int win_warps = 4;              // PENT_OPT_WINDOW_WARPS (0: off)
  int win_omax = 0;               // overlap rows reserved per window side (window rows / 8)
  int64_t win_cap = 0;            // windows the workspace holds
  int64_t nwin = 0;               // windows of the current factorisation (0: none)
  int win_even = 1;               // every windowed system starts at an even row
  std::vector<int32_t> wsys32;    // the other systems, bucket order
  std::vector<F32Bucket> wbuckets;
  std::vector<cudaStream_t> side; // extra streams so that bucket launches overlap
  std::vector<cudaEvent_t> ev;    // fork/join events
  std::vector<cudaStream_t> pipe; // slices of pent_solve_host_batch (copy in, solve, copy out)
  std::vector<cudaEvent_t> pev;   // their fork/join events
  std::vector<cudaEvent_t> sev;   // per-slice hand-over events (copied in, solved)
  // workspace regions
  Region r_info, r_perm, r_off, r_n, r_goff, r_glen, r_sigma, r_fwd, r_bwd, r_scr, r_fac32, r_sig32, r_foff, r_shape,
      r_sys32, r_adi, r_cmap, r_swU, r_swE, r_pck, r_pcc, r_pcbase, r_pcnum, r_pcmap, r_pU, r_pE, r_per, r_psinv,
      r_pg, r_rhs, r_psinv32, r_urec, r_kscale, r_uwin, r_win, r_whalo, r_wsys32, r_gover, r_win64, r_side64,
      r_halo64, r_icst, r_ik, r_lover, r_sbase, r_sfwd, r_sbwd, r_swin, r_sgs, r_swg;
  size_t ws_bytes = 0;
  // binding / state
  unsigned char* ws = nullptr;
  cudaStream_t stream = nullptr;
  bool bound = false;
  int factored = 0;  // 0 none, 1 general band, 2 hyperdiffusion
  // step-graph cache: (x, nsteps, max_refine, settings version) -> exec, at most kMaxGraphs
  // entries; the least recently launched is destroyed to make room (an exec still running
  // is freed by the runtime once it completes)
  using GraphKey = std::tuple<const void*, int64_t, int, int64_t>;
  struct GraphEntry {
    cudaGraphExec_t exec;
    uint64_t used;
  };
  std::map<GraphKey, GraphEntry> graphs;
  uint64_t graph_clock = 0;
  // ADI: the parameters this (shared-matrix) plan was factored for by adi_plans_factor
  bool adi_ready = false;
  double adi_gamma = 0.0, adi_dt = 0.0, adi_dx = 0.0, adi_sigma = 0.0;
  cudaGraphExec_t find_graph(const GraphKey& k) {
    auto it = graphs.find(k);
    if (it == graphs.end()) return nullptr;
    it->second.used = ++graph_clock;
    return it->second.exec;
  }
  void add_graph(const GraphKey& k, cudaGraphExec_t exec) {
    while (graphs.size() >= (size_t)PENT_MAX_CACHED_GRAPHS) {
      auto lru = graphs.begin();
      for (auto it = graphs.begin(); it != graphs.end(); ++it)
        if (it->second.used < lru->second.used) lru = it;
      cudaGraphExecDestroy(lru->second.exec);
      graphs.erase(lru);
    }
    graphs[k] = GraphEntry{exec, ++graph_clock};
  }

  template <class T>
  T* at(const Region& r) const {
    return reinterpret_cast<T*>(ws + r.off);
  }
  DevPlan dev() const {
    DevPlan P;
    P.batch = batch;
    P.ngroups = ngroups;
    P.shared = shared ? 1 : 0;
    P.n_shared = shared ? n_uniform : 0;
    P.perm = at<int32_t>(r_perm);
    P.off = at<int64_t>(r_off);
    P.n = at<int32_t>(r_n);
    P.goff = at<int64_t>(r_goff);
    P.glen = at<int32_t>(r_glen);
    P.info = at<unsigned long long>(r_info);
    return P;
  }
  // Hyperdiffusion factors of per-system matrices use the constant-epsilon records.
  F64Factors f64() const {
    F64Factors F{at<double>(r_fwd), at<double>(r_bwd), (factored == 2 && !shared) ? at<double>(r_sigma) : nullptr};
    if (factored == 2 && !shared && f64_interior && interior_valid && r_ik.bytes > 1) {
      F.icst = at<double2>(r_icst);
      F.ik = at<int32_t>(r_ik);
    }
    return F;
  }
  F64Part part() const {
    F64Part X;
    X.ck = at<int32_t>(r_pck);
    X.cc = at<int32_t>(r_pcc);
    X.cbase = at<int64_t>(r_pcbase);
    X.cnum = at<int32_t>(r_pcnum);
    X.cmap = at<double>(r_pcmap);
    X.U = at<double2>(r_pU);
    X.E = at<double2>(r_pE);
    return X;
  }
  PerArgs per() const {
    PerArgs A;
    A.batch = batch;
    A.n = n_uniform;
    A.m = n_uniform - 2;
    A.shared = shared ? 1 : 0;
    const int64_t plane = A.m * (shared ? 1 : batch);
    double* base = at<double>(r_per);
    double** planes[9] = {&A.ia, &A.bb, &A.ee, &A.ga, &A.de, &A.z0, &A.z1, &A.w0, &A.w1};
    for (int k = 0; k < 9; ++k) *planes[k] = base + k * plane;
    A.sinv = at<double>(r_psinv);
    A.gscr = at<double>(r_pg);
    A.info = at<unsigned long long>(r_info);
    return A;
  }
  F32Tables f32() const {
    F32Tables T;
    T.n = at<int32_t>(r_n);
    T.off = at<int64_t>(r_off);
    T.foff = at<int64_t>(r_foff);
    T.sig2 = at<float2>(r_sig32);
    T.sigma = at<double>(r_sigma);
    T.fac = at<float>(r_fac32);
    T.info = at<unsigned long long>(r_info);
    T.psinv = periodic ? at<float4>(r_psinv32) : nullptr;
    return T;
  }
  void drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();
  }
  void drop_streams() {
    for (auto e : ev) cudaEventDestroy(e);
    for (auto st : side) cudaStreamDestroy(st);
    for (auto e : pev) cudaEventDestroy(e);
    for (auto e : sev) cudaEventDestroy(e);
    for (auto st : pipe) cudaStreamDestroy(st);
    ev.clear();
    side.clear();
    pev.clear();
    sev.clear();
    pipe.clear();
  }
};

namespace {

pent_status cuda_status(cudaError_t e) { return e == cudaSuccess ? PENT_OK : PENT_ECUDA; }

using Shape = pent_plan::Shape;

// FP32 CTA shape for n rows with L rows per thread.  Up to 512 threads: one CTA
// of the fewest warps that cover n.  Beyond: a cluster of up to 8 CTAs of
// exactly cw warps (4 or 8), else of up to 8 CTAs with as few warps each (at
// most 16) as cover n.  On GB300, 8-warp clusters solve
// 6,144-16,384-row systems in 0.020-0.024 ms per million rows against 0.028-0.030
// for 16-warp ones (three CTAs resident per SM instead of one); up to 4,096 rows
// one CTA of up to 16 warps beats a cluster (0.018 against 0.024).
bool shape_with_rows(int64_t n, int L, Shape* sh, int cw = 8) {
  const int64_t t = (n + L - 1) / L;  // threads needed
  if (t <= 512) { *sh = Shape{L, (int)((t + 31) / 32), 1}; return true; }
  if (cw < 16) {
    const int64_t C = (t + 32 * cw - 1) / (32 * cw);
    if (C <= 8) { *sh = Shape{L, cw, (int)C}; return true; }
  }
  const int64_t C = (t + 511) / 512;
  if (C > 8) return false;
  *sh = Shape{L, (int)((t + 32 * C - 1) / (32 * C)), (int)C};
  return true;
}

// Built-in FP32 shape: 8 rows per thread (4 for the shortest systems).
// Padding is below 256 rows per system.
bool default_shape(int64_t n, Shape* sh, int cw) {
  if (n <= 128) { *sh = Shape{4, 1, 1}; return true; }
  return shape_with_rows(n, 8, sh, cw);
}

// Shape for a requested number of threads per system (32 W, W <= 16, or
// 512 C, C <= 8) and rows per thread (4 or 8; 0: the fewer that covers n).
bool shape_for_threads(int64_t n, int64_t tps, int rpt, Shape* sh) {
  if (tps < 32 || tps % 32) return false;
  int C = 1;
  if (tps > 512) {
    if (tps % 512) return false;
    C = (int)(tps / 512);
    if (C > 8) return false;
  }
  const int W = (int)(tps / (32 * C));
  if (W > 16) return false;
  for (int L : {4, 8}) {
    if (rpt && L != rpt) continue;
    if ((int64_t)32 * W * C * L >= n) { *sh = Shape{L, W, C}; return true; }
  }
  return false;
}

const pent_plan::Rule* find_rule(const pent_plan* p, int prec, int64_t n) {
  for (const auto& r : p->rules)
    if (r.prec == prec && r.lo <= n && n <= r.hi) return &r;
  return nullptr;
}

// Shape of an n-row system: options, then the tune cache, then the built-in rule.
bool choose_shape(const pent_plan* p, int64_t n, Shape* sh) {
  if (p->tps_override) return shape_for_threads(n, p->tps_override, (int)p->rpt_override, sh);
  if (p->rpt_override) return shape_with_rows(n, (int)p->rpt_override, sh, p->cluster_warps);
  if (const pent_plan::Rule* r = find_rule(p, PENT_F32_REFINE, n))
    return r->b ? shape_for_threads(n, r->b, r->a, sh) : shape_with_rows(n, r->a, sh, p->cluster_warps);
  return default_shape(n, sh, p->cluster_warps);
}

// Read a tune cache (format in pentbatch.h).  False for an unreadable file or
// a malformed line.
bool parse_tune_cache(const char* path, std::vector<pent_plan::Rule>* out) {
  std::ifstream in(path);
  if (!in) return false;
  std::string line;
  while (std::getline(in, line)) {
    const size_t h = line.find('#');
    if (h != std::string::npos) line.resize(h);
    std::istringstream ls(line);
    std::string kind;
    if (!(ls >> kind)) continue;  // blank or comment
    pent_plan::Rule r{};
    long long lo, hi, a, b;
    if (!(ls >> lo >> hi >> a >> b)) return false;
    std::string extra;
    if (ls >> extra) return false;
    if (lo < 1 || hi < lo) return false;
    if (kind == "f32") {
      if ((a != 4 && a != 8) || b < 0 || (b && (b % 32 || b > 4096))) return false;
      r.prec = PENT_F32_REFINE;
    } else if (kind == "f64") {
      if ((a != 2 && a != 4 && a != 8) || b < 1 || b > 8) return false;
      r.prec = PENT_F64;
    } else {
      return false;
    }
    r.lo = lo;
    r.hi = hi;
    r.a = (int)a;
    r.b = (int)b;
    out->push_back(r);
  }
  return true;
}

// Groups whose longest system has at least this many rows are solved by the
// partitioned kernels: a thread-per-system walk takes time proportional to its
// length, about 0.3 us per row on GB300, while the whole batch streams at
// about 64 bytes per row at ~6 TB/s; a group is cut into chunks when its walk
// would outlast the batch, and never below 2048 rows (where the doubled
// arithmetic of the partitioned passes costs more than it hides) -- unless the
// batch has fewer than 1024 groups of 32 systems (under about 7 warps per SM
// of a GB300), when the walks alone cannot hide their latency and chunks pay
// from 512 rows on (4,096 systems of 1024 rows: 0.25 against 0.44 ms a solve).
int64_t part_threshold(const pent_plan* p) {
  if (p->shared || p->part_rows == 0) return INT64_MAX;
  if (p->part_rows > 0) return p->part_rows;
  const int64_t floor_rows = p->ngroups < 1024 ? 512 : 2048;
  return std::max<int64_t>(floor_rows, p->rows / 28000);
}

// FP64 launches: groups (longest first) in runs of equal unroll / block warps,
// the long groups in partitioned runs with their chunk lists.
void build_f64_runs(pent_plan* p) {
  p->runs.clear();
  p->pck.clear();
  p->pcc.clear();
  p->pcnum.assign(p->ngroups, 0);
  p->pcbase.assign(p->ngroups, 0);
  p->pchunks = 0;
  auto knobs = [&](int64_t len) {
    if (p->f64_explicit) return std::make_pair(p->unroll, p->block_warps);
    if (const pent_plan::Rule* r = find_rule(p, PENT_F64, len)) return std::make_pair(r->a, r->b);
    // built-in: the GB300 tuning at 2^26 rows (tune_gb300.txt): a group of long systems is
    // bound by the latency of its own serial walk, so it keeps 8 rows of loads in flight
    return len > 1024 ? std::make_pair(8, 1) : std::make_pair(4, 2);
  };
  if (p->shared) {
    // one broadcast record block: a row's only per-lane loads are f and g, and one-warp CTAs spread
    // the batch over the most SMs (65,536 x 1024 on GB300: unroll 4 one warp 0.65 ms a step,
    // two to four warps 0.70-0.77 ms, unroll 8 0.98 ms)
    const auto kb = p->f64_explicit ? std::make_pair(p->unroll, p->block_warps) : std::make_pair(4, 1);
    p->runs.push_back({0, p->ngroups, kb.first, kb.second, false, 0, 0});
    return;
  }
  const int64_t thr = part_threshold(p);
  for (int64_t k = 0; k < p->ngroups; ++k) {
    const bool part = p->gmax[k] >= thr;
    const auto kb = part ? std::make_pair(0, 0) : knobs(p->gmax[k]);
    if (part) {
      const int nch = (int)((p->glen[k] + kLongChunk - 1) / kLongChunk);
      p->pcbase[k] = p->pchunks;
      p->pcnum[k] = nch;
      for (int c = 0; c < nch; ++c) {
        p->pck.push_back((int32_t)k);
        p->pcc.push_back(c);
      }
      p->pchunks += nch;
    }
    auto& b = p->runs;
    if (!b.empty() && b.back().part == part && b.back().unroll == kb.first && b.back().bw == kb.second) {
      b.back().g1 = k + 1;
      b.back().c1 = p->pchunks;
    } else {
      const int64_t c0 = part ? p->pcbase[k] : p->pchunks;
      b.push_back({k, k + 1, kb.first, kb.second, part, c0, p->pchunks});
    }
  }
}

// Windows of an n-row system, R rows each with O overlap rows (multiples of 8, 4 O <= R): the
// first covers rows [0, R) and keeps [0, R - O); each next one starts O rows before the first
// row not yet kept and keeps R - 2 O rows; the last ends at row n and keeps the rest.  Writes
// (first row, rows, first kept, end kept) relative to the window per window while cap lasts
// and returns the count; 0 if n <= R (one CTA solves the system) or the sizes do not qualify.
int64_t window_layout(int64_t n, int R, int O, int32_t* out4, int64_t cap) {
  if (n <= R || R <= 0 || R % 8 || O <= 0 || O % 8 || 4 * O > R) return 0;
  int64_t k = 0;
  auto emit = [&](int64_t w0, int64_t m, int64_t o0, int64_t o1) {
    if (out4 && k < cap) {
      out4[4 * k] = (int32_t)w0;
      out4[4 * k + 1] = (int32_t)m;
      out4[4 * k + 2] = (int32_t)o0;
      out4[4 * k + 3] = (int32_t)o1;
    }
    ++k;
  };
  emit(0, R, 0, R - O);
  int64_t a = R - O;  // first row not yet kept
  while (n - a > R - O) {
    emit(a - O, R, O, R - O);
    a += R - 2 * O;
  }
  emit(a - O, n - a + O, O, n - a + O);
  return k;
}

// System windows of a system of np row pairs, windows of Rp pairs with Op pairs of overlap
// (0 < 4 Op <= Rp, or Op = 0 for systems of one window): three int32 per window {q0, k0, k1},
// walking pairs [q0, min(q0 + Rp, np)) and keeping [k0, k1).  The first window starts at pair 0
// and keeps [0, Rp - Op); each next one starts Op pairs before the first pair not yet kept and
// keeps Rp - 2 Op; the last starts at np - Rp, so it walks Rp pairs too and ends at the system's
// end, and keeps the rest (at least Op pairs from its start).  Returns the count.
int64_t swin_layout(int64_t np, int Rp, int Op, int32_t* out3, int64_t cap) {
  int64_t k = 0;
  auto emit = [&](int64_t q0, int64_t k0, int64_t k1) {
    if (out3 && k < cap) {
      out3[3 * k] = (int32_t)q0;
      out3[3 * k + 1] = (int32_t)k0;
      out3[3 * k + 2] = (int32_t)k1;
    }
    ++k;
  };
  if (np <= 0) return 0;
  if (np <= Rp) {
    emit(0, 0, np);
    return k;
  }
  if (Op <= 0 || 4 * Op > Rp) return 0;
  emit(0, 0, Rp - Op);
  int64_t a = Rp - Op;  // first pair not yet kept
  while (np - a > Rp - Op) {
    emit(a - Op, a, a + Rp - 2 * Op);
    a += Rp - 2 * Op;
  }
  emit(np - Rp, a, np);
  return k;
}

bool build_f32_shapes(pent_plan* p) {
  const int64_t nfac = p->shared ? 1 : p->batch;
  p->shape.assign(nfac, Shape{0, 0, 0});
  p->foff.assign(nfac, 0);
  int64_t acc = 0;
  for (int64_t s = 0; s < nfac; ++s) {
    const int64_t n = p->n[s];
    if (!choose_shape(p, n, &p->shape[s])) return false;
    p->foff[s] = acc;
    const Shape& sh = p->shape[s];
    const int planes = p->periodic ? 4 : 2;  // periodic blocks also hold Z = E^{-1} k
    acc += (int64_t)planes * 32 * sh.W * sh.C * sh.L / 4;
  }
  p->fac_float4 = acc;
  // buckets: systems grouped by shape, longest shapes first
  std::map<Shape, std::vector<int32_t>> groups;
  for (int64_t s = 0; s < p->batch; ++s) groups[p->shape[p->shared ? 0 : s]].push_back((int32_t)s);
  std::vector<std::pair<Shape, std::vector<int32_t>>> order(groups.begin(), groups.end());
  std::sort(order.begin(), order.end(), [](const auto& a, const auto& b) {
    return (int64_t)a.first.W * a.first.C * a.first.L > (int64_t)b.first.W * b.first.C * b.first.L;
  });
  p->sys32.clear();
  p->buckets.clear();
  for (auto& kv : order) {
    F32Bucket b;
    b.L = kv.first.L;
    b.W = kv.first.W;
    b.C = kv.first.C;
    b.first = (int64_t)p->sys32.size();
    b.count = (int64_t)kv.second.size();
    b.even_offsets = 1;
    for (int32_t s : kv.second) {
      if (p->off[s] & 1) b.even_offsets = 0;
      p->sys32.push_back(s);
    }
    p->buckets.push_back(b);
  }
  p->threads_per_system = p->shared || p->uniform ? 32 * p->shape[0].W * p->shape[0].C : 0;
  return true;
}

void layout(pent_plan* p) {
  size_t cur = 0;
  auto take = [&](Region& r, size_t bytes) {
    r.off = cur;
    r.bytes = bytes;
    cur = align_up(cur + std::max<size_t>(bytes, 1));
  };
  const int64_t nfac = p->shared ? 1 : p->batch;
  take(p->r_info, kInfoWords * sizeof(unsigned long long));
  take(p->r_perm, (size_t)p->ngroups * kWarp * sizeof(int32_t));
  take(p->r_off, (size_t)p->batch * sizeof(int64_t));
  take(p->r_n, (size_t)p->batch * sizeof(int32_t));
  take(p->r_goff, (size_t)p->ngroups * sizeof(int64_t));
  take(p->r_glen, (size_t)p->ngroups * sizeof(int32_t));
  take(p->r_sigma, (size_t)nfac * sizeof(double));
  if (p->periodic && p->precision == PENT_F64) {
    // Navon's reduction: nine interleaved planes of the reduced matrix, S^{-1}, and g
    const int64_t m = p->n_uniform - 2;
    take(p->r_per, (size_t)9 * m * nfac * sizeof(double));
    take(p->r_psinv, (size_t)4 * nfac * sizeof(double));
    take(p->r_pg, (size_t)m * p->batch * sizeof(double));
    p->ws_bytes = cur;
    return;
  }
  if (p->precision == PENT_F64) {
    const int64_t frows = p->shared ? p->n_uniform : p->grows;
    const int64_t lanes = p->shared ? 1 : kWarp;
    take(p->r_fwd, (size_t)frows * 3 * lanes * sizeof(double));
    take(p->r_bwd, (size_t)frows * 2 * lanes * sizeof(double));
    take(p->r_scr, (size_t)p->grows * kWarp * sizeof(double));
    take(p->r_pck, (size_t)p->pchunks * sizeof(int32_t));
    take(p->r_pcc, (size_t)p->pchunks * sizeof(int32_t));
    take(p->r_pcbase, (size_t)p->ngroups * sizeof(int64_t));
    take(p->r_pcnum, (size_t)p->ngroups * sizeof(int32_t));
    take(p->r_pcmap, (size_t)p->pchunks * 8 * kWarp * sizeof(double));
    take(p->r_pU, (size_t)p->pchunks * kWarp * 2 * sizeof(double));
    take(p->r_pE, (size_t)p->pchunks * kWarp * 2 * sizeof(double));
    // right-hand sides of pent_step_batch for the partitioned groups (their chunked solve reads f)
    take(p->r_rhs, (size_t)(p->pchunks > 0 ? p->rows : 0) * sizeof(double));
    // windows of long groups (hyperdiffusion factorisations): as many as the largest overlap needs
    p->win64_cap = 0;
    p->win64_omax = 0;
    if (!p->shared && p->win64_rows > 0) {
      p->win64_omax = p->win64_rows / 8;
      for (int64_t k = 0; k < p->ngroups; ++k)
        p->win64_cap += window_layout(p->glen[k], p->win64_rows, p->win64_omax, nullptr, 0);
    }
    // system windows: room for every system of a group longer than one window
    p->swin_cap = p->srec_pairs = p->srec_maxpairs = 0;
    if (p->win64_cap > 0 && p->win64_form == 1) {
      // a system window keeps its rows at least O from each cut: room for O up to a quarter of it
      p->win64_omax = p->win64_rows / 4;
      const int Rp = p->win64_rows / 2;
      for (int64_t k = 0; k < p->ngroups; ++k) {
        if (p->glen[k] <= p->win64_rows) continue;
        for (int j = 0; j < kWarp; ++j) {
          const int32_t s = p->perm[(size_t)(k * kWarp + j)];
          if (s < 0) continue;
          const int64_t np = (p->n[s] + 1) / 2;
          p->srec_pairs += np;
          p->srec_maxpairs = std::max(p->srec_maxpairs, np);
          p->swin_cap += swin_layout(np, Rp, p->win64_omax / 2, nullptr, 0);
        }
      }
      p->win64_cap = 0;  // the group windows' room is not needed
    }
    const size_t wpairs = (size_t)p->win64_cap * (p->win64_omax / 2) * kWarp;  // double2 per window side
    // interior records per group lane (hyperdiffusion factorisations)
    take(p->r_icst, (size_t)(p->shared ? 0 : p->ngroups * kWarp) * 4 * sizeof(double2));
    take(p->r_ik, (size_t)(p->shared ? 0 : p->ngroups * kWarp) * sizeof(int32_t));
    const bool any_win = p->win64_cap > 0 || p->swin_cap > 0;
    take(p->r_gover, (size_t)(any_win ? p->ngroups : 0) * sizeof(int32_t));
    take(p->r_lover, (size_t)(p->swin_cap > 0 ? p->ngroups * kWarp : 0) * sizeof(int32_t));
    take(p->r_sbase, (size_t)(p->swin_cap > 0 ? p->ngroups * kWarp : 0) * sizeof(int64_t));
    take(p->r_swg, (size_t)(p->swin_cap > 0 ? p->ngroups : 0) * sizeof(int32_t));
    take(p->r_sfwd, (size_t)p->srec_pairs * 3 * sizeof(double2));
    take(p->r_sbwd, (size_t)p->srec_pairs * 2 * sizeof(double2));
    take(p->r_swin, (size_t)p->swin_cap * sizeof(int4));
    take(p->r_sgs, (size_t)((p->swin_cap + kWarp - 1) / kWarp) * kWarp * (p->win64_rows / 2) * sizeof(double2));
    take(p->r_win64, (size_t)p->win64_cap * sizeof(int4));
    take(p->r_side64, wpairs * 2 * sizeof(double));
    take(p->r_halo64, wpairs * 4 * sizeof(double));
  } else {
    take(p->r_fac32, (size_t)p->fac_float4 * 4 * sizeof(float));
    take(p->r_sig32, (size_t)nfac * 2 * sizeof(float));
    take(p->r_foff, (size_t)nfac * sizeof(int64_t));
    take(p->r_shape, (size_t)nfac * sizeof(int32_t));
    take(p->r_sys32, (size_t)p->batch * sizeof(int32_t));
    if (p->periodic) take(p->r_psinv32, (size_t)nfac * 4 * sizeof(float));
    if (!p->periodic) {  // interior-constant kernel: per factor block record, per system field scale
      take(p->r_urec, (size_t)nfac * kURecFloat4 * sizeof(float4));
      take(p->r_kscale, (size_t)p->batch * sizeof(int32_t));
      // windows: as many as the largest overlap could need (the count grows with the overlap)
      p->win_cap = 0;
      p->win_omax = 0;
      if (p->win_warps > 0) {
        const int R = 256 * p->win_warps;
        p->win_omax = R / 8;
        for (int64_t s = 0; s < p->batch; ++s) p->win_cap += window_layout(p->n[s], R, p->win_omax, nullptr, 0);
      }
      take(p->r_uwin, (size_t)nfac * sizeof(int2));
      take(p->r_win, (size_t)p->win_cap * sizeof(int4));
      take(p->r_whalo, (size_t)p->win_cap * 2 * p->win_omax * sizeof(double));
      take(p->r_wsys32, (size_t)(p->win_cap > 0 ? p->batch : 0) * sizeof(int32_t));
    }
  }
  // ADI scratch, for shared-matrix plans whose batch is the number of columns of
  // a sweep: a full field (rows doubles), the partial sums of the sweep
  // (ceil(batch / 32) per chunk) and the mean; the chunk maps of the
  // factorisation and the per-(chunk, column) affine parts / entering states.
  if (p->shared) {
    const int64_t nch = (p->n_uniform + kAdiChunk - 1) / kAdiChunk;
    take(p->r_adi, (size_t)(p->rows + nch * ((p->batch + 31) / 32) + 8) * sizeof(double));
    take(p->r_cmap, (size_t)nch * 8 * sizeof(double));
    take(p->r_swU, (size_t)nch * p->batch * 2 * sizeof(double));
    take(p->r_swE, (size_t)nch * p->batch * 2 * sizeof(double));
  }
  p->ws_bytes = cur;
}

// Launch count(i) for i = 0..n-1: on the plan's stream alone, or spread over
// the plan's side streams (forked from and joined back to the plan's stream
// with events, which also works inside a stream capture).  first_alone: launch
// 0 (the windows, the bulk of the work) keeps the plan's stream to itself and
// the others share the side streams, so none waits behind it.
template <class F>
cudaError_t fork_join(pent_plan* p, size_t n, F launch, bool first_alone = false) {
  const int ns = (int)p->side.size();
  cudaError_t e = cudaSuccess;
  if (ns == 0 || n < 2) {
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) e = launch(i, p->stream);
    return e;
  }
  e = cudaEventRecord(p->ev[0], p->stream);
  for (int k = 0; k < ns && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(p->side[k], p->ev[0], 0);
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
    cudaStream_t st = (i % (ns + 1) == 0) ? p->stream : p->side[i % (ns + 1) - 1];
    if (first_alone) st = i == 0 ? p->stream : p->side[(i - 1) % ns];
    e = launch(i, st);
  }
  for (int k = 0; k < ns && e == cudaSuccess; ++k) {
    e = cudaEventRecord(p->ev[1 + k], p->side[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->stream, p->ev[1 + k], 0);
  }
  return e;
}

}  // namespace

extern "C" {

const char* pent_version(void) { return "0.1.0"; }

const char* pent_status_string(pent_status s) {
  switch (s) {
    case PENT_OK: return "ok";
    case PENT_EINVAL: return "invalid argument";
    case PENT_ESINGULAR: return "zero or non-finite pivot";
    case PENT_ENOCONV: return "refinement did not converge";
    case PENT_ECUDA: return "CUDA error";
    case PENT_ENOTFACTORED: return "not factored";
    case PENT_ENOTBOUND: return "no workspace bound";
  }
  return "unknown status";
}

pent_status pent_plan_create(pent_plan** out, int64_t batch, const int64_t* n_per_system, int64_t n_uniform,
                             int shared_matrix, pent_precision precision, const char* tune_cache) {
  if (!out) return PENT_EINVAL;
  *out = nullptr;
  if (batch < 1 || batch > (int64_t)INT32_MAX) return PENT_EINVAL;
  if (precision != PENT_F64 && precision != PENT_F32_REFINE) return PENT_EINVAL;
  if (shared_matrix && n_per_system) return PENT_EINVAL;
  pent_plan* p = new pent_plan();
  if (tune_cache && !parse_tune_cache(tune_cache, &p->rules)) {
    delete p;
    return PENT_EINVAL;
  }
  p->batch = batch;
  p->shared = shared_matrix != 0;
  p->precision = precision;
  p->n.resize(batch);
  for (int64_t s = 0; s < batch; ++s) {
    const int64_t v = n_per_system ? n_per_system[s] : n_uniform;
    if (v < 1 || v > (int64_t)INT32_MAX) {
      delete p;
      return PENT_EINVAL;
    }
    p->n[s] = v;
  }
  p->off.assign(batch + 1, 0);
  for (int64_t s = 0; s < batch; ++s) p->off[s + 1] = p->off[s] + p->n[s];
  p->rows = p->off[batch];
  p->uniform = std::all_of(p->n.begin(), p->n.end(), [&](int64_t v) { return v == p->n[0]; });
  p->n_uniform = p->uniform ? p->n[0] : 0;
  // groups of 32 systems, longest first (stable), so a warp's lanes walk similar lengths
  p->ngroups = (batch + kWarp - 1) / kWarp;
  std::vector<int32_t> order(batch);
  std::iota(order.begin(), order.end(), 0);
  if (!p->uniform)
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return p->n[x] > p->n[y]; });
  p->perm.assign(p->ngroups * kWarp, -1);
  for (int64_t q = 0; q < batch; ++q) p->perm[q] = order[q];
  p->goff.resize(p->ngroups);
  p->glen.resize(p->ngroups);
  p->gmax.resize(p->ngroups);
  int64_t acc = 0;
  for (int64_t k = 0; k < p->ngroups; ++k) {
    int64_t mx = 0;
    for (int l = 0; l < kWarp; ++l) {
      const int32_t s = p->perm[k * kWarp + l];
      if (s >= 0) mx = std::max(mx, p->n[s]);
    }
    p->gmax[k] = mx;
    if (!p->shared) mx += (mx & 1);  // per-system records are stored in row pairs
    p->goff[k] = acc;
    p->glen[k] = (int32_t)mx;
    acc += mx;
  }
  p->grows = acc;
  build_f64_runs(p);
  if (precision == PENT_F32_REFINE) {
    if (!build_f32_shapes(p)) {
      delete p;
      return PENT_EINVAL;
    }
  }
  layout(p);
  *out = p;
  return PENT_OK;
}

size_t pent_plan_workspace_bytes(const pent_plan* p) { return p ? p->ws_bytes : 0; }

int64_t pent_window_layout(int64_t n, int window_rows, int overlap, int32_t* h_out4, int64_t cap) {
  return window_layout(n, window_rows, overlap, h_out4, cap < 0 ? 0 : cap);
}

int64_t pent_system_window_layout(int64_t n, int window_rows, int overlap, int32_t* h_out3, int64_t cap) {
  if (n <= 0 || window_rows <= 0 || window_rows % 2 || overlap < 0 || overlap % 2) return 0;
  const int64_t np = (n + 1) / 2;
  const int64_t cnt = swin_layout(np, window_rows / 2, overlap / 2, h_out3, cap < 0 ? 0 : cap);
  for (int64_t i = 0; h_out3 && i < std::min(cnt, cap); ++i) {
    h_out3[3 * i] *= 2;
    h_out3[3 * i + 1] *= 2;
    h_out3[3 * i + 2] = (int32_t)std::min<int64_t>(2 * (int64_t)h_out3[3 * i + 2], n);
  }
  return cnt;
}

pent_status pent_plan_bind(pent_plan* p, void* ws, void* stream) {
  if (!p || !ws) return PENT_EINVAL;
  if (((uintptr_t)ws) % kAlign) return PENT_EINVAL;
  p->drop_graphs();
  p->ws = static_cast<unsigned char*>(ws);
  p->stream = static_cast<cudaStream_t>(stream);
  std::vector<int32_t> n32(p->batch);
  for (int64_t s = 0; s < p->batch; ++s) n32[s] = (int32_t)p->n[s];
  cudaError_t e = cudaSuccess;
  auto up = [&](const Region& r, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpy(p->ws + r.off, src, bytes, cudaMemcpyHostToDevice);
  };
  up(p->r_perm, p->perm.data(), p->perm.size() * sizeof(int32_t));
  up(p->r_off, p->off.data(), (size_t)p->batch * sizeof(int64_t));
  up(p->r_n, n32.data(), n32.size() * sizeof(int32_t));
  up(p->r_goff, p->goff.data(), p->goff.size() * sizeof(int64_t));
  up(p->r_glen, p->glen.data(), p->glen.size() * sizeof(int32_t));
  const unsigned long long init[kInfoWords] = {kInfoNone, 0, 0, 0};
  up(p->r_info, init, sizeof(init));
  if (p->precision == PENT_F64 && !p->shared) {
    up(p->r_pck, p->pck.data(), p->pck.size() * sizeof(int32_t));
    up(p->r_pcc, p->pcc.data(), p->pcc.size() * sizeof(int32_t));
    up(p->r_pcbase, p->pcbase.data(), p->pcbase.size() * sizeof(int64_t));
    up(p->r_pcnum, p->pcnum.data(), p->pcnum.size() * sizeof(int32_t));
  }
  if (p->precision == PENT_F32_REFINE) {
    std::vector<int32_t> shp(p->shape.size());
    for (size_t k = 0; k < shp.size(); ++k)
      shp[k] = (32 * p->shape[k].W * p->shape[k].C) | (p->shape[k].L << 16);
    up(p->r_foff, p->foff.data(), p->foff.size() * sizeof(int64_t));
    up(p->r_shape, shp.data(), shp.size() * sizeof(int32_t));
    up(p->r_sys32, p->sys32.data(), p->sys32.size() * sizeof(int32_t));
  }
  // side streams (and fork/join events) so that several launches of one solve overlap
  p->drop_streams();
  const bool win64 = p->win64_cap > 0 || p->swin_cap > 0;
  const size_t nlaunch = p->precision == PENT_F64 ? p->runs.size() + (win64 ? 1 : 0)
                                                 : p->buckets.size() + (p->win_cap > 0 ? 1 : 0);
  // with windows the other launches share the side streams among themselves (fork_join's first_alone)
  const size_t maxside = (p->win_cap > 0 || win64) ? 6 : 3;
  const int nside = (int)std::min<size_t>(maxside, nlaunch > 1 ? nlaunch - 1 : 0);
  for (int k = 0; k < nside && e == cudaSuccess; ++k) {
    cudaStream_t ss;
    e = cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking);
    if (e == cudaSuccess) p->side.push_back(ss);
  }
  for (int k = 0; k < 2 * nside + 1 && e == cudaSuccess; ++k) {
    cudaEvent_t ee;
    e = cudaEventCreateWithFlags(&ee, cudaEventDisableTiming);
    if (e == cudaSuccess) p->ev.push_back(ee);
  }
  // streams of the host-resident pipeline (pent_solve_host_batch)
  constexpr int kPipe = 3;
  for (int k = 0; k < kPipe && e == cudaSuccess; ++k) {
    cudaStream_t ss;
    e = cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking);
    if (e == cudaSuccess) p->pipe.push_back(ss);
  }
  for (int k = 0; k < kPipe + 1 && e == cudaSuccess; ++k) {
    cudaEvent_t ee;
    e = cudaEventCreateWithFlags(&ee, cudaEventDisableTiming);
    if (e == cudaSuccess) p->pev.push_back(ee);
  }
  if (e != cudaSuccess) return PENT_ECUDA;
  p->bound = true;
  p->factored = 0;
  p->nwin = 0;
  p->nwin64 = 0;
  return PENT_OK;
}

pent_status pent_plan_set_option(pent_plan* p, int key, int64_t value) {
  if (!p) return PENT_EINVAL;
  switch (key) {
    case PENT_OPT_THREADS_PER_SYSTEM: {
      // changes the factor layout and the workspace size: only before binding
      if (p->bound) return PENT_EINVAL;
      if (p->precision == PENT_F64) return value == 1 ? PENT_OK : PENT_EINVAL;
      const int64_t keep = p->tps_override;
      p->tps_override = value;
      if (!build_f32_shapes(p)) {
        p->tps_override = keep;
        build_f32_shapes(p);
        return PENT_EINVAL;
      }
      layout(p);
      return PENT_OK;
    }
    case PENT_OPT_PARTITION_ROWS:
      if (p->bound || p->precision != PENT_F64) return PENT_EINVAL;
      if (value < -1) return PENT_EINVAL;
      p->part_rows = value;
      build_f64_runs(p);
      layout(p);
      return PENT_OK;
    case PENT_OPT_PERIODIC:
      if (p->bound || (value != 0 && value != 1)) return PENT_EINVAL;
      if (value == 1 && (!p->uniform || p->n_uniform < 5)) return PENT_EINVAL;
      p->periodic = value == 1;
      if (p->precision == PENT_F32_REFINE && !build_f32_shapes(p)) {
        p->periodic = false;
        build_f32_shapes(p);
        return PENT_EINVAL;
      }
      layout(p);
      return PENT_OK;
    case PENT_OPT_CLUSTER_WARPS: {
      if (p->bound || p->precision == PENT_F64) return PENT_EINVAL;
      if (value != 4 && value != 8 && value != 16) return PENT_EINVAL;
      const int keep = p->cluster_warps;
      p->cluster_warps = (int)value;
      if (!build_f32_shapes(p)) {
        p->cluster_warps = keep;
        build_f32_shapes(p);
        return PENT_EINVAL;
      }
      layout(p);
      return PENT_OK;
    }
    case PENT_OPT_ROWS_PER_THREAD: {
      if (p->bound) return PENT_EINVAL;
      if (p->precision == PENT_F64) return PENT_EINVAL;
      if (value != 0 && value != 4 && value != 8) return PENT_EINVAL;
      const int64_t keep = p->rpt_override;
      p->rpt_override = value;
      if (!build_f32_shapes(p)) {
        p->rpt_override = keep;
        build_f32_shapes(p);
        return PENT_EINVAL;
      }
      layout(p);
      return PENT_OK;
    }
    case PENT_OPT_RESIDUAL:
      if (value != PENT_RESIDUAL_FF && value != PENT_RESIDUAL_F64) return PENT_EINVAL;
      p->residual = (int)value;
      ++p->cfg_version;  // the kernels a step graph launches depend on it
      p->drop_graphs();
      return PENT_OK;
    case PENT_OPT_BLOCK_WARPS:
      if (value < 1 || value > 8) return PENT_EINVAL;
      p->block_warps = (int)value;
      p->f64_explicit = true;
      build_f64_runs(p);
      ++p->cfg_version;
      p->drop_graphs();
      return PENT_OK;
    case PENT_OPT_UNROLL:
      if (value != 2 && value != 4 && value != 8) return PENT_EINVAL;
      p->unroll = (int)value;
      p->f64_explicit = true;
      build_f64_runs(p);
      ++p->cfg_version;
      p->drop_graphs();
      return PENT_OK;
    case PENT_OPT_FP64_INTERIOR:
      if (p->precision != PENT_F64 || (value != 0 && value != 1)) return PENT_EINVAL;
      p->f64_interior = value == 1;
      ++p->cfg_version;
      p->drop_graphs();
      return PENT_OK;
    case PENT_OPT_PERSISTENT:
      if (p->periodic || (value != 0 && value != 1)) return PENT_EINVAL;
      p->persistent = value == 1;
      ++p->cfg_version;  // the launches a step graph holds depend on it
      p->drop_graphs();
      return PENT_OK;
    case PENT_OPT_WINDOW_ROWS:
      // changes the workspace size: only before binding
      if (p->bound || p->precision != PENT_F64 || p->periodic || p->shared) return PENT_EINVAL;
      if (value != 0 && (value < 256 || value > 16384 || value % 64)) return PENT_EINVAL;
      p->win64_rows = (int)value;
      layout(p);
      return PENT_OK;
    case PENT_OPT_WINDOW_FORM:
      // changes the workspace size: only before binding
      if (p->bound || p->precision != PENT_F64 || (value != 0 && value != 1)) return PENT_EINVAL;
      p->win64_form = (int)value;
      layout(p);
      return PENT_OK;
    case PENT_OPT_WINDOW_WARPS:
      // changes the workspace size: only before binding
      if (p->bound || p->precision != PENT_F32_REFINE || p->periodic) return PENT_EINVAL;
      if (value != 0 && !solve32w_supported((int)value)) return PENT_EINVAL;
      p->win_warps = (int)value;
      layout(p);
      return PENT_OK;
    case PENT_OPT_FP32_KERNEL:
      if (p->precision != PENT_F32_REFINE || (value != 0 && value != 1)) return PENT_EINVAL;
      p->f32_kernel = (int)value;
      ++p->cfg_version;
      p->drop_graphs();
      return PENT_OK;
    case PENT_OPT_REFINE_TOL_LOG2:
      if (value < 1 || value > 60) return PENT_EINVAL;
      p->tol_log2 = (int)value;
      ++p->cfg_version;
      p->drop_graphs();
      return PENT_OK;
  }
  return PENT_EINVAL;
}

pent_status pent_plan_get_option(const pent_plan* p, int key, int64_t* value) {
  if (!p || !value) return PENT_EINVAL;
  switch (key) {
    case PENT_OPT_THREADS_PER_SYSTEM: *value = p->threads_per_system; return PENT_OK;
    case PENT_OPT_RESIDUAL: *value = p->residual; return PENT_OK;
    case PENT_OPT_BLOCK_WARPS: *value = p->block_warps; return PENT_OK;
    case PENT_OPT_REFINE_TOL_LOG2: *value = p->tol_log2; return PENT_OK;
    case PENT_OPT_UNROLL: *value = p->unroll; return PENT_OK;
    case PENT_OPT_ROWS_PER_THREAD: *value = p->rpt_override; return PENT_OK;
    case PENT_OPT_PARTITION_ROWS: *value = p->part_rows; return PENT_OK;
    case PENT_OPT_PERIODIC: *value = p->periodic ? 1 : 0; return PENT_OK;
    case PENT_OPT_CLUSTER_WARPS: *value = p->cluster_warps; return PENT_OK;
    case PENT_OPT_FP32_KERNEL: *value = p->f32_kernel; return PENT_OK;
    case PENT_OPT_CACHED_GRAPHS: *value = (int64_t)p->graphs.size(); return PENT_OK;
    case PENT_OPT_WINDOW_WARPS: *value = p->win_warps; return PENT_OK;
    case PENT_OPT_WINDOWS: *value = p->precision == PENT_F64 ? p->nwin64 : p->nwin; return PENT_OK;
    case PENT_OPT_WINDOW_ROWS: *value = p->win64_rows; return PENT_OK;
    case PENT_OPT_PERSISTENT: *value = p->persistent ? 1 : 0; return PENT_OK;
    case PENT_OPT_FP64_INTERIOR: *value = p->f64_interior ? 1 : 0; return PENT_OK;
    case PENT_OPT_WINDOW_FORM: *value = p->win64_form; return PENT_OK;
  }
  return PENT_EINVAL;
}

pent_status pent_plan_system_config(const pent_plan* p, int64_t system, int64_t* a, int64_t* b) {
  if (!p || !a || !b || system < 0 || system >= p->batch) return PENT_EINVAL;
  if (p->periodic) {  // one thread per system, no tuned settings
    *a = 1;
    *b = 1;
    return PENT_OK;
  }
  if (p->precision == PENT_F32_REFINE) {
    const auto& sh = p->shape[p->shared ? 0 : system];
    *a = sh.L;
    *b = 32 * sh.W * sh.C;
    return PENT_OK;
  }
  // the group holding the system (sorted position q = group * 32 + lane)
  int64_t k = 0;
  if (!p->shared) {
    const auto it = std::find(p->perm.begin(), p->perm.end(), (int32_t)system);
    k = (int64_t)(it - p->perm.begin()) / kWarp;
  }
  for (const auto& r : p->runs)
    if (r.g0 <= k && k < r.g1) {
      *a = r.part ? 0 : r.unroll;
      *b = r.part ? kLongChunk : r.bw;
      return PENT_OK;
    }
  return PENT_EINVAL;
}

static pent_status reset_info(pent_plan* p) {
  // memsets only, so the reset is asynchronous and capture-safe
  cudaError_t e = cudaMemsetAsync(p->at<unsigned char>(p->r_info), 0x7f, sizeof(unsigned long long), p->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(p->at<unsigned char>(p->r_info) + sizeof(unsigned long long), 0,
                        (kInfoWords - 1) * sizeof(unsigned long long), p->stream);
  return cuda_status(e);
}

// Windows for the current factorisation: every system longer than one window CTA whose overlap
// (from k_uplan32) fits the reserved room, and whose head of non-constant factors ends before its
// second window starts, is cut into windows; the others keep their buckets.  The overlaps are
// read back, which waits for the plan's stream; under a stream capture no windows are built.
static cudaError_t build_windows(pent_plan* p) {
  const int64_t nprev = p->nwin;
  p->nwin = 0;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(p->stream, &cs);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusNone) {
    if (nprev) ++p->cfg_version;
    return cudaSuccess;
  }
  const int64_t nfac = p->shared ? 1 : p->batch;
  std::vector<int2> kw((size_t)nfac);
  e = cudaMemcpyAsync(kw.data(), p->at<int2>(p->r_uwin), (size_t)nfac * sizeof(int2), cudaMemcpyDeviceToHost,
                      p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);  // also: no solve still reads the old windows
  if (e != cudaSuccess) return e;
  const int R = 256 * p->win_warps;
  std::vector<int32_t> win, geo;  // four int32 per window
  std::vector<char> windowed((size_t)p->batch, 0);
  int even = 1;
  for (int64_t s = 0; s < p->batch; ++s) {
    const int64_t n = p->n[s];
    if (n <= R) continue;
    const int64_t ms = p->shared ? 0 : s;
    const int K = kw[ms].x, O = kw[ms].y;
    if (p->shape[ms].L != 8 || O <= 0 || O > p->win_omax || K > R - 2 * O) continue;
    const int64_t cnt = window_layout(n, R, O, nullptr, 0);
    geo.resize((size_t)(4 * cnt));
    window_layout(n, R, O, geo.data(), cnt);
    for (int64_t k = 0; k < cnt; ++k) {
      win.push_back((int32_t)s);
      win.push_back(geo[4 * k]);
      win.push_back(geo[4 * k + 1] | (O << 16));
      win.push_back(0);
    }
    windowed[s] = 1;
    if (p->off[s] & 1) even = 0;
  }
  const int64_t nw = (int64_t)win.size() / 4;
  if (nw > p->win_cap) return cudaErrorInvalidValue;  // not reached: the room is sized for the largest overlap
  p->wsys32.clear();
  p->wbuckets.clear();
  for (const F32Bucket& b : p->buckets) {
    F32Bucket q = b;
    q.first = (int64_t)p->wsys32.size();
    q.count = 0;
    q.even_offsets = 1;
    for (int64_t i = b.first; i < b.first + b.count; ++i) {
      const int32_t sy = p->sys32[i];
      if (windowed[sy]) continue;
      p->wsys32.push_back(sy);
      ++q.count;
      if (p->off[sy] & 1) q.even_offsets = 0;
    }
    if (q.count) p->wbuckets.push_back(q);
  }
  if (nw > 0) {
    e = cudaMemcpy(p->at<int4>(p->r_win), win.data(), (size_t)nw * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !p->wsys32.empty())
      e = cudaMemcpy(p->at<int32_t>(p->r_wsys32), p->wsys32.data(), p->wsys32.size() * sizeof(int32_t),
                     cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  p->nwin = nw;
  p->win_even = even;
  if (nw || nprev) ++p->cfg_version;  // step graphs hold the launches of the old layout
  return cudaSuccess;
}

// Launch settings (unroll, warps per CTA) of the FP64 windows: those a group of one window's rows
// takes (options, then the tune cache, then the built-in rule of build_f64_runs).
static std::pair<int, int> win64_knobs(const pent_plan* p) {
  const int R = p->win64_rows;
  if (p->f64_explicit) return {p->unroll, std::min(p->block_warps, 4)};
  if (const pent_plan::Rule* rl = find_rule(p, PENT_F64, R)) return {rl->a, std::min(rl->b, 4)};
  return R > 1024 ? std::make_pair(8, 1) : std::make_pair(4, 2);
}

// Windows of long groups for an FP64 hyperdiffusion factorisation: the groups longer than one
// window of every run whose such groups all have an overlap (k_overlap64) within the reserved
// room are walked in windows; the rest of each run is kept (a partitioned run keeps the chunks
// of its remaining groups).  The overlaps are read back, which waits for the plan's stream; under
// a stream capture no windows are built.
//
// System windows (PENT_OPT_WINDOW_FORM 1) of the windowed groups: every system of such a group is
// laid out with its own overlap (lover, by group lane), the systems taken in the order of their
// rows in the caller's layout (so are their windows and their records' copies), and the records
// are copied into the per-system layout.  Sets nwin64.
static cudaError_t build_system_windows(pent_plan* p, const std::vector<char>& windowed,
                                        const std::vector<int32_t>& lover) {
  const int Rp = p->win64_rows / 2;
  std::vector<int64_t> sbase((size_t)p->ngroups * kWarp, -1);
  std::vector<int32_t> wg, geo;
  std::vector<std::pair<int64_t, int64_t>> sys;  // (first row in the caller's layout, group lane)
  for (int64_t k = 0; k < p->ngroups; ++k) {
    if (!windowed[k]) continue;
    wg.push_back((int32_t)k);
    for (int j = 0; j < kWarp; ++j) {
      const int32_t s = p->perm[(size_t)(k * kWarp + j)];
      if (s >= 0) sys.push_back({p->off[s], k * kWarp + j});
    }
  }
  // systems, their windows and their records in the order of the caller's rows
  std::stable_sort(sys.begin(), sys.end());
  std::vector<int4> win;
  int64_t acc = 0;
  for (const auto& sg : sys) {
    const int64_t gl = sg.second;
    const int32_t s = p->perm[(size_t)gl];
    const int64_t np = (p->n[s] + 1) / 2;
    const int Op = lover[(size_t)gl] / 2;
    const int64_t cnt = swin_layout(np, Rp, Op, nullptr, 0);
    if (cnt <= 0) return cudaErrorInvalidValue;  // not reached: windowed groups have their overlaps in range
    geo.resize((size_t)(3 * cnt));
    swin_layout(np, Rp, Op, geo.data(), cnt);
    for (int64_t i = 0; i < cnt; ++i) win.push_back(make_int4((int)gl, geo[3 * i], geo[3 * i + 1], geo[3 * i + 2]));
    sbase[(size_t)gl] = acc;
    acc += np;
  }
  if ((int64_t)win.size() > p->swin_cap || acc > p->srec_pairs) return cudaErrorInvalidValue;  // not reached
  cudaError_t e = cudaSuccess;
  if (!win.empty()) {
    e = cudaMemcpy(p->at<int4>(p->r_swin), win.data(), win.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->at<int64_t>(p->r_sbase), sbase.data(), sbase.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->at<int32_t>(p->r_swg), wg.data(), wg.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    F64Factors F = p->f64();
    F.sig = p->at<double>(p->r_sigma);
    if (e == cudaSuccess)
      e = launch_srec64(p->dev(), F, p->at<int32_t>(p->r_swg), (int64_t)wg.size(), p->srec_maxpairs,
                        p->at<int64_t>(p->r_sbase), p->at<double2>(p->r_sfwd), p->at<double2>(p->r_sbwd), p->stream);
  }
  p->nwin64 = (int64_t)win.size();
  return e;
}

static cudaError_t build_windows64(pent_plan* p) {
  const int64_t nprev = p->nwin64;
  p->nwin64 = 0;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(p->stream, &cs);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusNone) {
    if (nprev) ++p->cfg_version;
    return cudaSuccess;
  }
  F64Factors F = p->f64();
  F.sig = p->at<double>(p->r_sigma);
  const bool sysw = p->swin_cap > 0;
  e = launch_overlap64(p->dev(), F, p->win64_omax, p->at<int32_t>(p->r_gover),
                       sysw ? p->at<int32_t>(p->r_lover) : nullptr, p->stream);
  std::vector<int32_t> gover((size_t)p->ngroups), lover(sysw ? (size_t)p->ngroups * kWarp : 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(gover.data(), p->at<int32_t>(p->r_gover), gover.size() * sizeof(int32_t),
                        cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess && sysw)
    e = cudaMemcpyAsync(lover.data(), p->at<int32_t>(p->r_lover), lover.size() * sizeof(int32_t),
                        cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);  // also: no solve still reads the old windows
  if (e != cudaSuccess) return e;
  const int R = p->win64_rows;
  std::vector<int32_t> win, geo;
  // per run: its groups longer than one window are walked in windows only if every one of them
  // decays fast enough (so each run splits once at most: its groups are sorted longest first)
  std::vector<char> windowed((size_t)p->ngroups, 0);
  for (const auto& r : p->runs) {
    bool ok = true;
    for (int64_t k = r.g0; k < r.g1 && ok; ++k)
      if (p->glen[k] > R && (gover[k] <= 0 || gover[k] > p->win64_omax)) ok = false;
    for (int64_t k = r.g0; k < r.g1 && ok; ++k) windowed[k] = p->glen[k] > R;
  }
  if (sysw) {
    e = build_system_windows(p, windowed, lover);
    if (e != cudaSuccess) return e;
  }
  for (int64_t k = 0; k < p->ngroups && !sysw; ++k) {
    const int O = gover[k];
    if (!windowed[k]) continue;
    const int64_t cnt = window_layout(p->glen[k], R, O, nullptr, 0);
    geo.resize((size_t)(4 * cnt));
    window_layout(p->glen[k], R, O, geo.data(), cnt);
    for (int64_t j = 0; j < cnt; ++j) {
      win.push_back((int32_t)k);
      win.push_back(geo[4 * j]);
      win.push_back(geo[4 * j + 1] | (O << 16));
      win.push_back(0);
    }
    windowed[k] = 1;
  }
  const int64_t nw = sysw ? p->nwin64 : (int64_t)win.size() / 4;
  if (!sysw && nw > p->win64_cap) return cudaErrorInvalidValue;  // not reached: the room is sized for the largest overlap
  p->wruns.clear();
  for (const auto& r : p->runs) {
    for (int64_t g = r.g0; g < r.g1;) {
      if (windowed[g]) {
        ++g;
        continue;
      }
      int64_t h = g;
      while (h < r.g1 && !windowed[h]) ++h;
      pent_plan::F64Run q = r;
      q.g0 = g;
      q.g1 = h;
      if (r.part) {
        q.c0 = p->pcbase[g];
        q.c1 = p->pcbase[h - 1] + p->pcnum[h - 1];
      }
      p->wruns.push_back(q);
      g = h;
    }
  }
  if (nw > 0 && !sysw) {
    e = cudaMemcpy(p->at<int4>(p->r_win64), win.data(), (size_t)nw * sizeof(int4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  p->nwin64 = nw;
  if (nw || nprev) ++p->cfg_version;  // step graphs hold the launches of the old layout
  return cudaSuccess;
}

// windows = false (a refactorisation inside a solve): lay out no FP64 windows (the layout would wait
// for the stream on every call), dropping those of an earlier factorisation, and find no interior
// records (the walks then read every record).
static pent_status factor_common(pent_plan* p, const double* a, const double* b, const double* c, const double* d,
                                 const double* e, const double* sigma, bool windows = true) {
  if (!p) return PENT_EINVAL;
  if (!p->bound) return PENT_ENOTBOUND;
  p->drop_graphs();
  p->adi_ready = false;
  pent_status st = reset_info(p);
  if (st != PENT_OK) return st;
  const DevPlan P = p->dev();
  const int64_t nsig = p->shared ? 1 : p->batch;
  if (sigma && sigma != p->at<double>(p->r_sigma)) {
    cudaError_t err = cudaMemcpyAsync(p->at<double>(p->r_sigma), sigma, (size_t)nsig * sizeof(double),
                                      cudaMemcpyDeviceToDevice, p->stream);
    if (err != cudaSuccess) return PENT_ECUDA;
  }
  const double* sg = sigma ? p->at<double>(p->r_sigma) : nullptr;
  cudaError_t err;
  if (p->periodic && p->precision == PENT_F64) {
    err = launch_factor_periodic(p->per(), a, b, c, d, e, sg, p->stream);
  } else if (p->precision == PENT_F64) {
    F64Factors F = p->f64();
    F.sig = (sigma && !p->shared) ? sg : nullptr;
    err = launch_factor64(P, a, b, c, d, e, sg, F, p->stream);
    // chunk maps of a shared factorisation, for the partitioned sweeps of the ADI step
    if (err == cudaSuccess && p->shared) err = launch_chunk_maps(F, (int)p->n_uniform, p->at<double>(p->r_cmap), p->stream);
    // chunk maps of the partitioned groups
    if (err == cudaSuccess && p->pchunks > 0) err = launch_chunk_maps64(P, F, p->part(), 0, p->pchunks, p->stream);
    // interior records of the hyperdiffusion walks
    p->interior_valid = false;
    if (err == cudaSuccess && sigma && !p->shared && windows) {
      err = launch_interior64(P, F, p->at<double2>(p->r_icst), p->at<int32_t>(p->r_ik), p->stream);
      p->interior_valid = err == cudaSuccess;
    }
    // windows of the long groups (hyperdiffusion records); a general band keeps the runs
    if (err == cudaSuccess && (p->win64_cap > 0 || p->swin_cap > 0)) {
      if (sigma && windows) {
        err = build_windows64(p);
      } else if (p->nwin64) {
        p->nwin64 = 0;
        ++p->cfg_version;
      }
    }
  }
  else if (p->periodic)
    err = launch_factor32_periodic(p->f32(), p->at<int32_t>(p->r_shape), p->shared ? 1 : p->batch, sg, p->stream);
  else {
    err = launch_factor32(p->f32(), p->at<int32_t>(p->r_shape), p->shared ? 1 : p->batch, sg, p->stream);
    if (err == cudaSuccess)
      err = launch_uplan32(p->f32(), p->at<int32_t>(p->r_shape), p->shared ? 1 : p->batch, p->at<float4>(p->r_urec),
                           p->at<int2>(p->r_uwin), p->stream);
    if (err == cudaSuccess && p->win_cap > 0) err = build_windows(p);
  }
  if (err != cudaSuccess) return PENT_ECUDA;
  p->factored = sigma ? 2 : 1;
  return PENT_OK;
}

pent_status pent_factor_batch(pent_plan* p, const double* a, const double* b, const double* c, const double* d,
                              const double* e) {
  const Range range("pent_factor_batch");
  if (!p || !a || !b || !c || !d || !e) return PENT_EINVAL;
  if (p->precision == PENT_F32_REFINE) return PENT_EINVAL;  // refinement needs the band in closed form (sigma)
  return factor_common(p, a, b, c, d, e, nullptr);
}

pent_status pent_factor_hyperdiff(pent_plan* p, const double* d_sigma) {
  const Range range("pent_factor_hyperdiff");
  if (!p || !d_sigma) return PENT_EINVAL;
  return factor_common(p, nullptr, nullptr, nullptr, nullptr, nullptr, d_sigma);
}

// True if the plan's FP32 solves with max_refine steps may take the interior-constant kernel
// (csrc/f32u.cu), single-CTA systems and windows alike.
static bool u_path(const pent_plan* p, int max_refine) {
  return p->precision == PENT_F32_REFINE && !p->periodic && p->residual == PENT_RESIDUAL_FF && p->f32_kernel == 0 &&
         max_refine <= 1;
}

// True if bucket b of an FP32 plan is solved by the interior-constant kernel.
static bool use_u(const pent_plan* p, const F32Bucket& b, int max_refine) {
  return u_path(p, max_refine) && solve32u_supported(b);
}

// True if the solve runs the long systems' windows (and the other systems' buckets).
static bool use_windows(const pent_plan* p, int max_refine) { return p->nwin > 0 && u_path(p, max_refine); }

// One FP32 solve of bucket b (systems [b.first, b.first + b.count) of the bucket order `sys`,
// the plan's order by default).  in_ff / out_ff: f / x of the bucket's systems hold scaled
// float pairs (interior-constant kernel only).
static cudaError_t f32_bucket(pent_plan* p, const F32Bucket& b, const double* f, double* x, int max_refine, int in_ff,
                              int out_ff, cudaStream_t st, const int32_t* sys = nullptr) {
  const F32Tables T = p->f32();
  if (!sys) sys = p->at<int32_t>(p->r_sys32);
  if (use_u(p, b, max_refine))
    return launch_solve32u(T, p->at<float4>(p->r_urec), p->at<int32_t>(p->r_kscale), sys, b, p->shared, f, x,
                           max_refine, in_ff, out_ff, st);
  if (in_ff || out_ff) return cudaErrorInvalidValue;
  return launch_solve32r(T, sys, b, p->shared, f, x, max_refine, p->residual == PENT_RESIDUAL_F64, p->tol_log2, st,
                         nullptr, nullptr, false, p->periodic);
}

static pent_status solve_launch(pent_plan* p, const double* f, double* x, int max_refine, int in_ff = 0,
                                int out_ff = 0) {
  cudaError_t err;
  if (p->periodic && p->precision == PENT_F64) {
    err = launch_solve_periodic(p->per(), f, x, nullptr, nullptr, false, p->stream);
  } else if (p->precision == PENT_F64) {
    const DevPlan P = p->dev();
    const F64Factors F = p->f64();
    double* gscr = p->at<double>(p->r_scr);
    const F64Part X = p->part();
    // windows of the long groups and the other groups' runs, each launch on its own branch
    const size_t nw = p->nwin64 > 0 ? 1 : 0;
    const std::vector<pent_plan::F64Run>& runs = nw ? p->wruns : p->runs;
    err = fork_join(p, runs.size() + nw, [&](size_t i, cudaStream_t st) {
      if (i < nw && p->swin_cap > 0)
        return launch_swin64(P, F, p->at<int4>(p->r_swin), p->nwin64, p->win64_rows, win64_knobs(p).first,
                             win64_knobs(p).second, p->at<double2>(p->r_sfwd), p->at<double2>(p->r_sbwd), p->at<int64_t>(p->r_sbase), f, x,
                             p->at<double2>(p->r_sgs), st);
      if (i < nw)
        return launch_solve64w(P, F, p->at<int4>(p->r_win64), p->nwin64, p->win64_omax, win64_knobs(p).first,
                               win64_knobs(p).second, f, x, gscr, p->at<double>(p->r_side64),
                               p->at<double>(p->r_halo64), p->persistent, st);
      const auto& r = runs[i - nw];
      if (r.part) return launch_solve64_part(P, F, X, f, x, gscr, r.g0, r.g1, r.c0, r.c1, st);
      return launch_solve64(P, F, f, x, gscr, r.bw, r.unroll, r.g0, r.g1, st);
    }, nw > 0);
  } else {
    if (p->periodic && p->residual == PENT_RESIDUAL_F64) return PENT_EINVAL;  // periodic: float-float residual
    // windows of the long systems (FP64 in and out: a window reads its neighbours' rows) and the
    // other systems' buckets, each launch on its own branch
    const bool w = use_windows(p, max_refine);
    const std::vector<F32Bucket>& bk = w ? p->wbuckets : p->buckets;
    const int32_t* sys = p->at<int32_t>(w ? p->r_wsys32 : p->r_sys32);
    const size_t nw = w ? 1 : 0;
    err = fork_join(p, bk.size() + nw, [&](size_t i, cudaStream_t st) {
      if (i < nw)
        return launch_solve32w(p->f32(), p->at<float4>(p->r_urec), p->at<int32_t>(p->r_shape), p->at<int4>(p->r_win),
                               p->nwin, p->win_warps, p->win_omax, p->shared, p->win_even, f, x,
                               p->at<double>(p->r_whalo), max_refine, p->persistent, st);
      const F32Bucket& b = bk[i - nw];
      const bool u = use_u(p, b, max_refine);
      return f32_bucket(p, b, f, x, max_refine, u && in_ff, u && out_ff, st, sys);
    }, nw > 0);
  }
  return cuda_status(err);
}

// `nsteps` repetitions of launch() on the plan's stream: captured once into a
// CUDA graph under `key` and replayed on later calls (plain launches on the
// legacy stream, which cannot be captured).
}  // extern "C"

template <class F>
static pent_status run_steps(pent_plan* p, const std::tuple<const void*, int64_t, int, int64_t>& key, int64_t nsteps,
                             F launch) {
  pent_status st = PENT_OK;
  if (p->stream == nullptr) {
    for (int64_t k = 0; k < nsteps && st == PENT_OK; ++k) st = launch();
    return st;
  }
  cudaGraphExec_t exec = p->find_graph(key);
  if (!exec) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PENT_ECUDA;
    for (int64_t k = 0; k < nsteps && st == PENT_OK; ++k) st = launch();
    cudaError_t e = cudaStreamEndCapture(p->stream, &g);
    if (st != PENT_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return st != PENT_OK ? st : PENT_ECUDA;
    }
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return PENT_ECUDA;
    p->add_graph(key, exec);
  }
  return cuda_status(cudaGraphLaunch(exec, p->stream));
}

extern "C" {

static pent_status check_solve(pent_plan* p, const void* f, const void* x, int max_refine) {
  if (!p || !f || !x || max_refine < 0) return PENT_EINVAL;
  if (!p->bound) return PENT_ENOTBOUND;
  if (!p->factored) return PENT_ENOTFACTORED;
  if ((((uintptr_t)f) | ((uintptr_t)x)) % sizeof(double)) return PENT_EINVAL;
  return PENT_OK;
}

pent_status pent_solve_batch(pent_plan* p, const double* f, double* x, int max_refine) {
  const Range range("pent_solve_batch");
  pent_status st = check_solve(p, f, x, max_refine);
  if (st != PENT_OK) return st;
  return solve_launch(p, f, x, max_refine);
}

}  // extern "C"

// Slices of one pent_solve_host_batch call at most (two hand-over events each; on
// GB300 the pipeline gains nothing beyond 16-24 slices).
constexpr int64_t kMaxSlices = 256;

// The device address of [h, h + bytes) when the whole range lies inside one
// page-locked host allocation that the GPU addresses directly (cudaHostAlloc,
// pinned tensors); nullptr for anything else (pageable memory, device memory,
// a range that runs past its allocation, a driver without the query).
static void* mapped_host_range(const void* h, size_t bytes) {
  using GetAttr = CUresult (*)(void*, CUpointer_attribute, CUdeviceptr);
  static const GetAttr get = []() -> GetAttr {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<GetAttr>(fn);
  }();
  if (!get || !h || bytes == 0) return nullptr;
  const CUdeviceptr hp = (CUdeviceptr)(uintptr_t)h;
  unsigned int type = 0;
  CUdeviceptr d = 0, start = 0;
  size_t size = 0;
  if (get(&type, CU_POINTER_ATTRIBUTE_MEMORY_TYPE, hp) != CUDA_SUCCESS || type != CU_MEMORYTYPE_HOST) return nullptr;
  if (get(&d, CU_POINTER_ATTRIBUTE_DEVICE_POINTER, hp) != CUDA_SUCCESS || d == 0) return nullptr;
  if (get(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, d) != CUDA_SUCCESS ||
      get(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, d) != CUDA_SUCCESS)
    return nullptr;
  if (d < start || d - start > size || bytes > size - (size_t)(d - start)) return nullptr;
  return reinterpret_cast<void*>((uintptr_t)d);
}

extern "C" {

pent_status pent_host_range_mapped(const void* h, size_t bytes) {
  return mapped_host_range(h, bytes) ? PENT_OK : PENT_EINVAL;
}

pent_status pent_solve_host_batch(pent_plan* p, const double* h_f, double* h_x, double* d_f, double* d_x,
                                  int nchunks, int max_refine) {
  const Range range("pent_solve_host_batch");
  if (!p || !h_f || !h_x || nchunks < 1) return PENT_EINVAL;
  if (!d_f && !d_x) {  // direct: the kernels read h_f and write h_x where they lie, over the host link
    if (p->precision != PENT_F32_REFINE || max_refine < 0) return PENT_EINVAL;
    if (!p->bound) return PENT_ENOTBOUND;
    if (!p->factored) return PENT_ENOTFACTORED;
    if ((((uintptr_t)h_f) | ((uintptr_t)h_x)) % sizeof(double)) return PENT_EINVAL;
    const size_t bytes = (size_t)p->rows * sizeof(double);
    const double* df = static_cast<const double*>(mapped_host_range(h_f, bytes));
    double* dx = static_cast<double*>(mapped_host_range(h_x, bytes));
    if (!df || !dx) return PENT_EINVAL;
    return solve_launch(p, df, dx, max_refine);
  }
  pent_status st = check_solve(p, d_f, d_x, max_refine);
  if (st != PENT_OK) return st;
  if ((((uintptr_t)h_f) | ((uintptr_t)h_x)) % sizeof(double)) return PENT_EINVAL;
  // slices of whole systems need one launch shape for the batch
  const bool f32_one = p->precision == PENT_F32_REFINE && !p->periodic && p->buckets.size() == 1 && p->uniform;
  const bool f64_one = p->precision == PENT_F64 && !p->periodic && p->runs.size() == 1 && !p->runs[0].part &&
                       p->uniform;
  int64_t units = f32_one ? p->batch : (f64_one ? p->ngroups : 1);  // slice granularity: systems or groups of 32
  const int K = (int)std::min<int64_t>(std::min<int64_t>(nchunks, units), kMaxSlices);
  auto sys_of = [&](int64_t u) { return f64_one ? std::min<int64_t>(u * kWarp, p->batch) : u; };
  cudaError_t e = cudaSuccess;
  if (K <= 1 || (!f32_one && !f64_one)) {  // one slice: copy in, solve, copy out on the plan's stream
    const size_t bytes = (size_t)p->rows * sizeof(double);
    e = cudaMemcpyAsync(d_f, h_f, bytes, cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) st = solve_launch(p, d_f, d_x, max_refine);
    if (e == cudaSuccess && st == PENT_OK) e = cudaMemcpyAsync(h_x, d_x, bytes, cudaMemcpyDeviceToHost, p->stream);
    return e != cudaSuccess ? PENT_ECUDA : st;
  }
  const int np = (int)p->pipe.size();
  while ((int)p->sev.size() < 2 * K && e == cudaSuccess) {  // per-slice hand-over events, kept by the plan
    cudaEvent_t ee;
    e = cudaEventCreateWithFlags(&ee, cudaEventDisableTiming);
    if (e == cudaSuccess) p->sev.push_back(ee);
  }
  if (e != cudaSuccess) return PENT_ECUDA;
  e = cudaEventRecord(p->pev[0], p->stream);
  for (int k = 0; k < np && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(p->pipe[k], p->pev[0], 0);
  const int64_t n = p->n_uniform;
  for (int c = 0; c < K && e == cudaSuccess; ++c) {
    const int64_t u0 = units * c / K, u1 = units * (c + 1) / K;
    const int64_t s0 = sys_of(u0), s1 = sys_of(u1);
    if (s1 <= s0) continue;
    // one stream per role: copies in, solves, copies out, each slice handed on by events, so
    // that neither copy direction waits behind the other in a stream's order
    cudaStream_t s_in = p->pipe[0], ss = p->pipe[1], s_out = p->pipe[2];
    const size_t off = (size_t)(s0 * n), bytes = (size_t)((s1 - s0) * n) * sizeof(double);
    e = cudaMemcpyAsync(d_f + off, h_f + off, bytes, cudaMemcpyHostToDevice, s_in);
    if (e == cudaSuccess) e = cudaEventRecord(p->sev[2 * c], s_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ss, p->sev[2 * c], 0);
    if (e != cudaSuccess) break;
    if (f32_one) {
      F32Bucket b = p->buckets[0];
      b.first += s0;
      b.count = s1 - s0;
      e = f32_bucket(p, b, d_f, d_x, max_refine, 0, 0, ss);
    } else {
      const auto& r = p->runs[0];
      e = launch_solve64(p->dev(), p->f64(), d_f, d_x, p->at<double>(p->r_scr), r.bw, r.unroll, u0, u1, ss);
    }
    if (e == cudaSuccess) e = cudaEventRecord(p->sev[2 * c + 1], ss);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, p->sev[2 * c + 1], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_x + off, d_x + off, bytes, cudaMemcpyDeviceToHost, s_out);
  }
  for (int k = 0; k < np && e == cudaSuccess; ++k) {
    e = cudaEventRecord(p->pev[1 + k], p->pipe[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->stream, p->pev[1 + k], 0);
  }
  return cuda_status(e);
}

pent_status pent_solve_steps(pent_plan* p, double* x, int64_t nsteps, int max_refine) {
  const Range range("pent_solve_steps");
  pent_status st = check_solve(p, x, x, max_refine);
  if (st != PENT_OK) return st;
  if (nsteps < 0) return PENT_EINVAL;
  if (nsteps == 0) return PENT_OK;
  const auto key = std::make_tuple((const void*)x, nsteps, max_refine, p->cfg_version);
  // FP32 plans on the interior-constant kernel keep the field as scaled float pairs between steps:
  // the first step reads FP64, the last writes FP64
  int64_t k = 0;
  return run_steps(p, key, nsteps, [&]() {
    const int in_ff = k > 0, out_ff = k + 1 < nsteps;
    ++k;
    return solve_launch(p, x, x, max_refine, in_ff, out_ff);
  });
}

// One pent_step_batch step on a no-flux FP64 plan: the fused right-hand side
// and solve for the thread-per-system runs; for partitioned runs the right-hand
// side is written out first, then solved by the chunked kernels.
static pent_status step_launch(pent_plan* p, const double* mu, const double* nu, double* C, int max_refine) {
  if (p->precision == PENT_F32_REFINE) {
    const F32Tables T = p->f32();
    const int32_t* sys = p->at<int32_t>(p->r_sys32);
    const cudaError_t err = fork_join(p, p->buckets.size(), [&](size_t i, cudaStream_t st) {
      return launch_solve32r(T, sys, p->buckets[i], p->shared, C, C, max_refine, 0, p->tol_log2, st, mu, nu, true,
                             p->periodic);
    });
    return cuda_status(err);
  }
  const DevPlan P = p->dev();
  const F64Factors F = p->f64();
  double* gscr = p->at<double>(p->r_scr);
  const F64Part X = p->part();
  double* frhs = p->at<double>(p->r_rhs);
  const cudaError_t err = fork_join(p, p->runs.size(), [&](size_t i, cudaStream_t st) {
    const auto& r = p->runs[i];
    if (r.part) {
      const cudaError_t e = launch_step_rhs(P, mu, nu, C, frhs, r.g0, r.g1, st);
      if (e != cudaSuccess) return e;
      return launch_solve64_part(P, F, X, frhs, C, gscr, r.g0, r.g1, r.c0, r.c1, st);
    }
    return launch_step64(P, F, mu, nu, C, gscr, r.bw, r.unroll, r.g0, r.g1, st);
  });
  return cuda_status(err);
}

pent_status pent_step_batch(pent_plan* p, const double* mu, const double* nu, double* C, int64_t nsteps,
                            int max_refine) {
  const Range range("pent_step_batch");
  pent_status st = check_solve(p, C, C, max_refine);
  if (st != PENT_OK) return st;
  if (nsteps < 0) return PENT_EINVAL;
  if ((((uintptr_t)mu) | ((uintptr_t)nu)) % sizeof(double)) return PENT_EINVAL;
  // no-flux plans: factors from sigma (pent_factor_hyperdiff); FP64 per-system, or FP32+refine with the
  // float-float residual
  if (!p->periodic && p->factored != 2) return PENT_EINVAL;
  if (!p->periodic && p->precision == PENT_F64 && p->shared) return PENT_EINVAL;
  if (p->precision == PENT_F32_REFINE && p->residual != PENT_RESIDUAL_FF) return PENT_EINVAL;
  if (nsteps == 0) return PENT_OK;
  auto launch = [&]() -> pent_status {
    if (p->periodic && p->precision == PENT_F64)
      return cuda_status(launch_solve_periodic(p->per(), C, C, mu, nu, true, p->stream));
    return step_launch(p, mu, nu, C, max_refine);
  };
  if (nsteps == 1) return launch();
  uint64_t h = 1469598103934665603ull;
  for (uint64_t v : {(uint64_t)(uintptr_t)mu, (uint64_t)(uintptr_t)nu, (uint64_t)p->cfg_version})
    h = (h ^ v) * 1099511628211ull;
  const auto key = std::make_tuple((const void*)C, nsteps, -2 - max_refine, (int64_t)(h & 0x7fffffffffffffffull));
  return run_steps(p, key, nsteps, launch);
}

pent_status pent_refactor_solve_hyperdiff(pent_plan* p, const double* d_sigma, const double* f, double* x) {
  const Range range("pent_refactor_solve_hyperdiff");
  if (!p || !d_sigma) return PENT_EINVAL;
  if (!p->bound) return PENT_ENOTBOUND;
  if (!f || !x || (((uintptr_t)f) | ((uintptr_t)x) | ((uintptr_t)d_sigma)) % sizeof(double)) return PENT_EINVAL;
  if (p->precision != PENT_F64 || p->periodic) return PENT_EINVAL;
  if (p->shared || p->pchunks > 0) {
    // one matrix for the batch, or groups solved in chunks: factor, then solve
    pent_status st = factor_common(p, nullptr, nullptr, nullptr, nullptr, nullptr, d_sigma, false);
    return st != PENT_OK ? st : solve_launch(p, f, x, 0);
  }
  pent_status st = reset_info(p);
  if (st != PENT_OK) return st;
  const DevPlan P = p->dev();
  F64Factors F = p->f64();
  F.sig = p->at<double>(p->r_sigma);
  if (p->factored != 2) p->drop_graphs();  // graphs cached for another record form
  double* gscr = p->at<double>(p->r_scr);
  cudaError_t err = fork_join(p, p->runs.size(), [&](size_t i, cudaStream_t s) {
    const auto& r = p->runs[i];
    return launch_refactor_solve64(P, F, d_sigma, f, x, gscr, r.bw, r.g0, r.g1, s);
  });
  // the records are new: their interior is not known (the walks read every record until the next
  // pent_factor_hyperdiff finds it; finding it here would cost about as much as the solve), and the
  // windows' overlaps were those of the old sigma
  p->interior_valid = false;
  if (err != cudaSuccess) return PENT_ECUDA;
  if (p->nwin64) {
    p->nwin64 = 0;
    ++p->cfg_version;
  }
  p->factored = 2;
  return PENT_OK;
}

pent_status pent_adjoint_solve_batch(pent_plan* p, const double* f, double* x, int max_refine) {
  const Range range("pent_adjoint_solve_batch");
  pent_status st = check_solve(p, f, x, max_refine);
  if (st != PENT_OK) return st;
  if (p->periodic) return PENT_EINVAL;
  // A = I + sigma D4 with the reflected D4 = D2N^2 is symmetric: A^{-T} f = A^{-1} f, by the
  // (faster, partitioned where the plan partitions) forward kernels and, for FP32+refine
  // plans, with their refinement
  if (p->factored == 2) return solve_launch(p, f, x, max_refine);
  if (p->precision != PENT_F64) return PENT_EINVAL;
  return cuda_status(
      launch_adjoint64(p->dev(), p->f64(), f, x, p->at<double>(p->r_scr), p->block_warps, p->stream));
}

pent_status pent_hyperdiff_sigma_grad(pent_plan* p, const double* mu, const double* x, double* g_sigma) {
  if (!p || !mu || !x || !g_sigma) return PENT_EINVAL;
  if (!p->bound) return PENT_ENOTBOUND;
  if (p->periodic) return PENT_EINVAL;  // the reduction reads only the plan's offsets: either precision
  return cuda_status(launch_sigma_grad(p->dev(), mu, x, g_sigma, p->stream));
}

pent_status pent_get_info(pent_plan* p, int64_t* bad_system, int64_t* bad_row, int* refine_steps_used) {
  if (!p) return PENT_EINVAL;
  if (!p->bound) return PENT_ENOTBOUND;
  unsigned long long h[kInfoWords];
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(h, p->at<unsigned long long>(p->r_info), sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return PENT_ECUDA;
  const bool bad = h[0] != kInfoNone;
  if (bad_system) *bad_system = bad ? (int64_t)(h[0] >> 32) : -1;
  if (bad_row) *bad_row = bad ? (int64_t)(h[0] & 0xffffffffull) : -1;
  if (refine_steps_used) *refine_steps_used = (int)h[1];
  if (bad) return PENT_ESINGULAR;
  if (h[2] & 1ull) return PENT_ENOCONV;
  return PENT_OK;
}

pent_status pent_clear_info(pent_plan* p) {
  if (!p) return PENT_EINVAL;
  if (!p->bound) return PENT_ENOTBOUND;
  return reset_info(p);
}

void pent_plan_destroy(pent_plan* p) {
  if (!p) return;
  p->drop_graphs();
  p->drop_streams();
  delete p;
}

static pent_status adi_check(pent_plan* px, pent_plan* py, double* C, int64_t nx, int64_t ny, double gamma, double dt,
                             double dx, int max_refine) {
  if (!px || !py || !C || nx < 1 || ny < 1 || max_refine != 0) return PENT_EINVAL;
  if (!(gamma > 0.0) || !(dt > 0.0) || !(dx > 0.0)) return PENT_EINVAL;
  if (nx > INT32_MAX || ny > INT32_MAX) return PENT_EINVAL;
  if (!px->bound || !py->bound) return PENT_ENOTBOUND;
  if (px->factored != 2 || py->factored != 2) return PENT_ENOTFACTORED;
  if (px->precision != PENT_F64 || py->precision != PENT_F64 || !px->shared || !py->shared) return PENT_EINVAL;
  if (px->periodic || py->periodic) return PENT_EINVAL;
  if (px->batch != ny || px->n_uniform != nx || py->batch != nx || py->n_uniform != ny) return PENT_EINVAL;
  if (px->stream != py->stream) return PENT_EINVAL;
  if (((uintptr_t)C) % sizeof(double)) return PENT_EINVAL;
  // the step's explicit part and its sweeps must use one scheme: both plans factored by
  // adi_plans_factor for exactly these (gamma, dt, dx)
  for (const pent_plan* q : {px, py})
    if (!q->adi_ready || q->adi_gamma != gamma || q->adi_dt != dt || q->adi_dx != dx) return PENT_EINVAL;
  return PENT_OK;
}

static pent_status adi_launch(pent_plan* px, pent_plan* py, double* C, int64_t nx, int64_t ny, double gamma, double dt,
                              double dx) {
  AdiArgs a;
  a.C = C;
  a.rhsT = px->at<double>(px->r_adi);
  a.W = px->at<double>(px->r_scr);
  a.parts = py->at<double>(py->r_adi) + nx * ny;
  const int64_t nchy = (ny + kAdiChunk - 1) / kAdiChunk;
  a.mean = a.parts + nchy * ((nx + 31) / 32);
  a.nx = (int)nx;
  a.ny = (int)ny;
  a.mu = dt / (dx * dx);
  a.sigma = px->adi_sigma;  // the sigma both plans were factored with
  a.sx = SweepArgs{px->f64(), px->at<double>(px->r_cmap), px->at<double2>(px->r_swU), px->at<double2>(px->r_swE)};
  a.sy = SweepArgs{py->f64(), py->at<double>(py->r_cmap), py->at<double2>(py->r_swU), py->at<double2>(py->r_swE)};
  return cuda_status(launch_adi_step(a, px->stream));
}

pent_status adi_plans_factor(pent_plan* px, pent_plan* py, double gamma, double dt, double dx) {
  const Range range("adi_plans_factor");
  if (!px || !py || px == py) return PENT_EINVAL;
  if (!(gamma > 0.0) || !(dt > 0.0) || !(dx > 0.0)) return PENT_EINVAL;
  for (const pent_plan* q : {px, py}) {
    if (!q->bound) return PENT_ENOTBOUND;
    if (q->precision != PENT_F64 || !q->shared || q->periodic) return PENT_EINVAL;
  }
  if (px->batch != py->n_uniform || py->batch != px->n_uniform || px->stream != py->stream) return PENT_EINVAL;
  const double sigma = gamma * dt / (dx * dx * dx * dx);  // Sec. 2.1: the fourth-order term's coefficient
  if (!std::isfinite(sigma) || !(sigma > 0.0)) return PENT_EINVAL;
  for (pent_plan* q : {px, py}) {
    // sigma into the plan's own slot by a kernel argument (asynchronous, capture-safe), then factor from it
    double* slot = q->at<double>(q->r_sigma);
    if (launch_fill(slot, sigma, 1, q->stream) != cudaSuccess) return PENT_ECUDA;
    const pent_status st = factor_common(q, nullptr, nullptr, nullptr, nullptr, nullptr, slot);
    if (st != PENT_OK) return st;
    q->adi_ready = true;
    q->adi_gamma = gamma;
    q->adi_dt = dt;
    q->adi_dx = dx;
    q->adi_sigma = sigma;
  }
  return PENT_OK;
}

pent_status adi_step_2d(pent_plan* px, pent_plan* py, double* C, int64_t nx, int64_t ny, double gamma, double dt,
                        double dx, int max_refine) {
  const Range range("adi_step_2d");
  pent_status st = adi_check(px, py, C, nx, ny, gamma, dt, dx, max_refine);
  if (st != PENT_OK) return st;
  return adi_launch(px, py, C, nx, ny, gamma, dt, dx);
}

pent_status adi_steps_2d(pent_plan* px, pent_plan* py, double* C, int64_t nx, int64_t ny, double gamma, double dt,
                         double dx, int max_refine, int64_t nsteps) {
  const Range range("adi_steps_2d");
  pent_status st = adi_check(px, py, C, nx, ny, gamma, dt, dx, max_refine);
  if (st != PENT_OK) return st;
  if (nsteps < 0) return PENT_EINVAL;
  if (nsteps == 0) return PENT_OK;
  if (px->stream == nullptr) {
    for (int64_t k = 0; k < nsteps && st == PENT_OK; ++k) st = adi_launch(px, py, C, nx, ny, gamma, dt, dx);
    return st;
  }
  // graphs of ADI steps are keyed by (C, nsteps, -1, hash of the parameters) in px's cache
  uint64_t h = 1469598103934665603ull;
  for (double v : {gamma, dt, dx}) {
    uint64_t b;
    std::memcpy(&b, &v, sizeof b);
    h = (h ^ b) * 1099511628211ull;
  }
  h ^= (uint64_t)(uintptr_t)py;
  const auto key = std::make_tuple((const void*)C, nsteps, -1, (int64_t)(h & 0x7fffffffffffffffull));
  cudaGraphExec_t exec = px->find_graph(key);
  if (!exec) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(px->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PENT_ECUDA;
    for (int64_t k = 0; k < nsteps && st == PENT_OK; ++k) st = adi_launch(px, py, C, nx, ny, gamma, dt, dx);
    cudaError_t e = cudaStreamEndCapture(px->stream, &g);
    if (st != PENT_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return st != PENT_OK ? st : PENT_ECUDA;
    }
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return PENT_ECUDA;
    px->add_graph(key, exec);
  }
  return cuda_status(cudaGraphLaunch(exec, px->stream));
}

}  // extern "C"
