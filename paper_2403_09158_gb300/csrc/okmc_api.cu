// Host side of the C ABI declared in include/okmc.h: handle life cycle, device
// memory under an optional budget, validation, and the order of kernel launches
// of each call.  All arithmetic of the method runs in the kernels of solve.cu
// and defects.cu; this file only marshals, validates and sequences.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <array>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <string>

#include <sys/stat.h>
#include <unistd.h>
#include <utility>
#include <vector>

#include "fft_reg.cuh"
#include "okmc_internal.cuh"

using namespace okmc;

namespace okmc {
template <class T> int pick_cluster(int H, int ny, size_t limit);
template <class T> int pick_tile(int ny, int nz, size_t limit);
template <class T, class Q> cudaError_t launch_plane_fwd(const Q* eps, C2<T>* spec, const PassCfg& c, cudaStream_t st);
template <class T> cudaError_t launch_plane_inv(const C2<T>* spec, T* sig, const PassCfg& c, cudaStream_t st);
template <class T> cudaError_t launch_pencil(C2<T>* spec, const PassCfg& c, cudaStream_t st);
cudaError_t launch_defect_setup(const okmc_defect* d, DefGeo* G, int nd, double h, cudaStream_t st);
cudaError_t launch_stencil_count(const DefGeo* G, int nd, int* nnz, long long* sumcnt, cudaStream_t st);
cudaError_t launch_dilate_count(const DefGeo* G, int nd, const int* ptr, const int* off, const uint8_t* cnt, int* ndil,
                                cudaStream_t st);
cudaError_t launch_dilate_fill(const DefGeo* G, int nd, const int* ptr, const int* off, const uint8_t* cnt,
                               const DilatedLists& dl, int* err, cudaStream_t st);
cudaError_t launch_stencil_fill(const DefGeo* G, int nd, const int* ptr, const long long* sumcnt, int* off, uint8_t* cnt,
                                double* alpha, int* err, cudaStream_t st);
template <class Q>
cudaError_t launch_voxelise(Q* eps, int3 n, const okmc_defect* d, const DefGeo* G, int nd, const int* ptr, const int* off,
                            const uint8_t* cnt, const double* alpha, double rq, double lim, int* err, cudaStream_t st);
template <class Q>
cudaError_t launch_apply_moves(Q* eps, int3 n, const DefGeo* G, int maxmoves, const int* ptr, const int* off,
                               const uint8_t* cnt, const double* alpha, const Move* moves, const DevState* stt, double rq,
                               double lim, int* err, int* dirty, cudaStream_t st);
cudaError_t launch_diff_positions(okmc_defect* d, const int* pos, int nd, Move* moves, DevState* stt, cudaStream_t st);
cudaError_t launch_gather_positions(const okmc_defect* d, int* pos, int nd, cudaStream_t st);
template <class Q, class T> cudaError_t launch_fixed_to_real(const Q* eps, T* out, size_t total, double q, cudaStream_t st);
template <class Q>
cudaError_t launch_wfields(Q* f, int3 n, const int* ptr, const int* off, const uint8_t* cnt, const WBatch& b, cudaStream_t st);
template <class QT>
cudaError_t launch_qtable(QT* out, const PassCfg& c, const QTypes& qt, cudaStream_t st);
template <class T>
cudaError_t launch_selfterm(const C2<T>* spec, const PassCfg& c, const WBatch& b, const T* qtab, const double2* phx,
                            const double2* phy, const double2* phz, double* partial, int nblocks, const double* alpha,
                            double pref, double* W, cudaStream_t st);
template <class T>
cudaError_t launch_energies(const T* sig, int3 n, const okmc_defect* d, const DefGeo* G, int nd, const int* ptr,
                            const int* off, const uint8_t* cnt, const double* alpha, const double* W, double pref,
                            int want_cand, const int* order, int nbig, double* E, double* Ec, RateArgs ra, const DilatedLists& dl,
                            cudaStream_t st);
// batched ensemble kernels (solve_fast.cu, defects.cu)
bool batch_edge_supported(int nx, int ny, int nz);
int pass_batch_grid(int pass, int n, int nitems);
cudaError_t launch_pass_batch(int pass, int n, const BatchRep* reps, const int2* items, int nitems, int grid, int slot0,
                              cudaStream_t st);
cudaError_t upload_batch_cfg(int slot0, const PassCfg* cfgs, int n, cudaStream_t st);
int batch_cfg_slots();
cudaError_t launch_energy_chunks_batch(const BatchRep* reps, const int2* items, int nitems, int grid, cudaStream_t st);
cudaError_t launch_energy_finish_batch(const BatchRep* reps, const int2* items, int nitems, int grid, cudaStream_t st);
template <class T>
cudaError_t launch_energy_chunks(const T* sig, int3 n, const okmc_defect* d, const DefGeo* G, int nd,
                                 const DilatedLists& dl, const ChunkArgs& ca, cudaStream_t st);
cudaError_t launch_energy_finish(const okmc_defect* d, const DefGeo* G, int nd, const DilatedLists& dl,
                                 const ChunkArgs& ca, const double* alpha, const double* W, double pref, double* E,
                                 double* Ec, RateArgs ra, cudaStream_t st);
cudaError_t launch_event_batch(const BatchRep* reps, int nrep, cudaStream_t st);
cudaError_t launch_moves_batch(const BatchRep* reps, int nrep, cudaStream_t st);
int energies_batch_grid();
cudaError_t launch_residence(okmc_defect* d, int nd, const double* rates, const double* rsum, int3 n, uint64_t seed,
                             Move* moves, DevState* stt, cudaStream_t st);
cudaError_t launch_fixed_dt(okmc_defect* d, const DefGeo* G, int nd, const double* rates, double nu0, double kT, int3 n,
                            uint64_t seed, Move* moves, DevState* stt, cudaStream_t st);
bool fast_solve_supported(const PassCfg& c);
cudaError_t launch_plane_fast(bool inverse, int variant, const void* in, void* out, const PassCfg& c, cudaStream_t st);
int plane_inv_variant_mask(const PassCfg& c);
int plane_fwd_variant_mask(const PassCfg& c);
template <class T, class QT>
cudaError_t launch_dipself(const C2<T>* spec, const PassCfg& c, const WBatch& b, const QT* qtab, const double2* phx,
                           const double2* phy, const double2* phz, double* partial, int nblocks, const double* alpha,
                           const DefGeo* G, double scale, double* D, cudaStream_t st);
template <class T>
cudaError_t launch_dipole_energies(const T* sig, int3 n, const okmc_defect* def, const DefGeo* G, const double* D, int nd,
                                   double h3, double* E, double* Ec, cudaStream_t st);
cudaError_t launch_pencil_fast(int variant, const C2<float>* in, C2<float>* out, const CUtensorMap* tin,
                               const CUtensorMap* tout, const PassCfg& c, cudaStream_t st);
int pencil_variant_mask(const PassCfg& c);
template <class T> int fdm_pencil_tile(int ny, int nz, size_t limit);
int shift_positions_per_pass();
template <class T>
cudaError_t launch_shift_energies(const C2<T>* spec_e, const C2<T>* spec_w, const PassCfg& c, const okmc_defect* def,
                                  const DefGeo* G, const double* alpha, int i, const double* X, int m, double h,
                                  double* partial, int nblocks, double* E, cudaStream_t st);
template <class T>
cudaError_t launch_point_dipole(const T* sig, int3 n, const int* pos, const double* P, int m, double C11, double C12,
                                double C44, double* E, int* err, cudaStream_t st);
template <class T, class Q>
cudaError_t launch_dislocation_eigenstrain(const double* pts, const int2* seg, const int* seg_line, int nseg,
                                           const int* first, const int* closed, const double* burgers, double* area,
                                           int nl, double ds_max, const PassCfg& c0, double h, int tw,
                                           unsigned long long* alpha_q, C2<T>* spec, Q* bg, double q, double qlim,
                                           int* err, cudaStream_t st);
}  // namespace okmc

namespace {
constexpr size_t kSmemLimit = 225 * 1024;
constexpr int kSelfBlocks = 608;

struct Pending {
  const char* name;
  cudaEvent_t a, b;
};

struct Status {
  int code;
  std::string msg;
};

int factor_ok(int n) {
  if (n < 16 || n > 512 || n % 16) return 0;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  while (n % 5 == 0) n /= 5;
  return n == 1;
}

template <class T>
void twiddles(std::vector<C2<T>>& out, int L, int count, double sign) {
  for (int k = 0; k < count; ++k) {
    const double ang = 2.0 * kPi * (double)k / (double)L;
    out.push_back(C2<T>{(T)std::cos(ang), (T)(sign * std::sin(ang))});
  }
}

// Twiddles exp(-2 pi i m / L), m < count, for the FP32 register-FFT passes.  Rounding
// cos and sin to nearest leaves |w| = 1 + d_m with d_m of either sign; a transform
// scales its output by the mean of the d_m it applies (weighted by how often it applies
// each twiddle), and for the tables of the solve that mean is a few 1e-9, a systematic
// error of the self term of every defect.  Each entry is therefore chosen among the
// FP32 pairs within two units in the last place of (cos, sin) whose phase error stays
// below 6e-8 rad, as the one that keeps the weighted running sum of d_m closest to
// zero (error diffusion): the table's weighted mean magnitude error then vanishes to
// within one entry's error over the table.  weight[m]: how often m is applied (empty:
// every entry once).
void balanced_twiddles(std::vector<C2<float>>& out, int L, int count, const std::vector<int>& weight) {
  double run = 0.0;
  for (int m = 0; m < count; ++m) {
    const double th = -2.0 * kPi * (double)m / (double)L;
    const double c = std::cos(th), s = std::sin(th);
    const int wgt = weight.empty() ? 1 : weight[m];
    C2<float> best{(float)c, (float)s};
    double best_d = (double)best.x * best.x + (double)best.y * best.y - 1.0, best_key = std::fabs(run + wgt * best_d);
    if (wgt > 0) {
      // the rounded values and their neighbours up to two units in the last place
      float cs[5], ss[5];
      cs[0] = (float)c;
      ss[0] = (float)s;
      float cu = cs[0], cd = cs[0], su = ss[0], sd = ss[0];
      for (int k = 1; k <= 2; ++k) {
        cs[2 * k - 1] = cu = std::nextafter(cu, 2.f);
        cs[2 * k] = cd = std::nextafter(cd, -2.f);
        ss[2 * k - 1] = su = std::nextafter(su, 2.f);
        ss[2 * k] = sd = std::nextafter(sd, -2.f);
      }
      for (float cc : cs)
        for (float sv : ss) {
          const double ph = c * ((double)sv - s) - s * ((double)cc - c);
          if (std::fabs(ph) > 6e-8) continue;
          const double d = (double)cc * cc + (double)sv * sv - 1.0;
          const double key = std::fabs(run + wgt * d);
          if (key < best_key) {
            best_key = key;
            best_d = d;
            best = C2<float>{cc, sv};
          }
        }
    }
    run += wgt * best_d;
    out.push_back(best);
  }
}

// How often the two-step register FFT of length L applies w_L^m between its steps
// (m = n1 k2, n1 < R1, 0 < k2 < R2).
std::vector<int> twiddle_use(int L) {
  std::vector<int> w(L, 0);
  int R1 = 0, R2 = 0;
  if (!reg_split(L, R1, R2)) return {};
  for (int n1 = 0; n1 < R1; ++n1)
    for (int k2 = 1; k2 < R2; ++k2) ++w[(n1 * k2) % L];
  return w;
}
}  // namespace

struct okmc_grid {
  okmc_grid_desc desc{};
  int n[3] = {0, 0, 0};
  int H = 0;
  size_t N = 0, P = 0;
  double h = 0, nu0 = 1e13;
  int prec = 0;
  cudaStream_t st = nullptr;
  size_t bytes = 0;
  std::vector<std::pair<void*, size_t>> allocs;
  void* eps = nullptr;
  void* sig = nullptr;
  void* spec = nullptr;
  void* spec2 = nullptr;  // fast path: Green operator output (spec keeps the plane transforms)
  // fast path: spec and spec2 as 2-D float tensors of 6 nz rows of 2 P floats, for the
  // TMA-staged pencil pass (valid when tm_ok)
  CUtensorMap tm_spec{}, tm_spec2{};
  bool tm_ok = false;
  int* d_dirty = nullptr;  // [6][nz] planes whose eigenstrain changed since their last transform
  void* tw = nullptr;
  void* ftw = nullptr;  // FP32 fields: twiddles with balanced magnitude errors, for the register-FFT passes
  double2* ph = nullptr;
  PassCfg cfg{};
  int nd = 0;
  okmc_defect* d_def = nullptr;
  DefGeo* d_geo = nullptr;
  int* d_ptr = nullptr;
  int* d_off = nullptr;
  uint8_t* d_cnt = nullptr;
  double* d_alpha = nullptr;
  long long* d_sumcnt = nullptr;
  int* d_nnz = nullptr;
  double* d_W = nullptr;
  double* d_D = nullptr;    // [nd][2][9] dipole self parts (int eps*) : sigma_i at the site centres
  double* d_dip = nullptr;  // [nd] dipole site energies, then [nd][8] candidate energies
  bool dip_valid = false;   // d_D holds the current defects' dipole self parts
  double* d_E = nullptr;
  double* d_Ec = nullptr;
  int* d_order = nullptr;  // defects by decreasing energy-list length (energies order)
  int nbig = 0;            // the first nbig of the order take a block each, the rest a warp
  double* d_rates = nullptr;
  double* d_rsum = nullptr;
  Move* d_moves = nullptr;
  DevState* d_state = nullptr;
  int* d_err = nullptr;
  int* d_pos = nullptr;
  double* d_partial = nullptr;
  int* d_dl = nullptr;                  // [4 nd]: start and end of each dilated candidate list
  int* d_doff = nullptr;                // dilated lists: packed offsets
  unsigned long long* d_dcnt = nullptr; // energy lists: eight candidate counts
  uint8_t* d_dscnt = nullptr;           // energy lists: site counts
  int* d_cdef = nullptr;                // energies by chunks: the defect of each chunk slot
  int* d_c0 = nullptr;                  // the first chunk slot of each defect
  double* d_cpart = nullptr;            // [nchunk][9] chunk sums
  int nchunk = 0;                       // chunk slots; 0: a defect has no energy list (per-defect kernel)
  void* d_bg = nullptr;     // [6][nz][ny][nx] fixed-point plastic strain of the dislocation lines (or none)
  std::vector<okmc_defect> h_def;
  bool sigma_valid = false;
  bool any_mobile = false;
  bool fast = false;  // FP32 register-FFT passes for this grid
  int variant[3] = {0, 0, 0};  // launch variant of the forward plane, pencil and inverse plane passes
  int avail[3] = {1, 1, 1};    // bit v: variant v exists for this grid
  long long solves = 0;
  std::string err;
  bool profiling = false;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> free_events;
  std::map<std::string, std::pair<double, long long>> prof;
  std::vector<std::string> prof_names;
  // captured step graphs, one per (mode, temperature)
  struct StepGraph {
    int mode;
    double T;
    cudaGraphExec_t exec;
  };
  std::vector<StepGraph> graphs;
  bool use_graphs = true;
  long long gen = 0;  // bumped by okmc_set_defects (device buffers may move)
};

struct okmc_batch {
  std::vector<okmc_grid*> grids;
  std::vector<long long> gens;
  std::vector<okmc_step_params> params;
  cudaStream_t st = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;
  std::string err;
  int mode = OKMC_BATCH_AUTO;  // requested form
  int used = 0;                // form of the current graph
  // batched kernels: replica records and work lists (planes, tiles, defects) on the device
  BatchRep* d_reps = nullptr;
  int2* d_items = nullptr;
  int slot0 = -1, nslots = 0;  // constant-memory slots of the replicas' pass configurations
};

// Constant-memory slots for the pass configurations of batched replicas, handed out to
// batches as contiguous ranges (first fit) and returned when a batch is rebuilt or destroyed.
std::mutex g_slot_mu;
std::vector<char> g_slot_used;

static int acquire_slots(int n) {
  std::lock_guard<std::mutex> lk(g_slot_mu);
  if ((int)g_slot_used.size() != batch_cfg_slots()) g_slot_used.assign(batch_cfg_slots(), 0);
  for (int s0 = 0; s0 + n <= (int)g_slot_used.size(); ++s0) {
    bool free_run = true;
    for (int k = 0; k < n && free_run; ++k) free_run = !g_slot_used[s0 + k];
    if (free_run) {
      for (int k = 0; k < n; ++k) g_slot_used[s0 + k] = 1;
      return s0;
    }
  }
  return -1;
}

static void release_slots(okmc_batch* b) {
  if (b->slot0 < 0) return;
  std::lock_guard<std::mutex> lk(g_slot_mu);
  for (int k = 0; k < b->nslots; ++k) g_slot_used[b->slot0 + k] = 0;
  b->slot0 = -1;
  b->nslots = 0;
}

namespace {

int fail(okmc_grid* g, int code, const std::string& m) {
  if (g) g->err = m;
  return code;
}
int cuda_fail(okmc_grid* g, cudaError_t e, const char* where) {
  return fail(g, OKMC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int dalloc(okmc_grid* g, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (g->desc.hbm_budget && g->bytes + bytes > g->desc.hbm_budget)
    return fail(g, OKMC_ENOMEM, "device allocation exceeds hbm_budget");
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(g, OKMC_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  g->allocs.push_back({*p, bytes});
  g->bytes += bytes;
  return OKMC_OK;
}
void dfree(okmc_grid* g, void* p) {
  if (!p) return;
  for (size_t k = 0; k < g->allocs.size(); ++k)
    if (g->allocs[k].first == p) {
      g->bytes -= g->allocs[k].second;
      g->allocs.erase(g->allocs.begin() + k);
      break;
    }
  cudaFree(p);
}

cudaEvent_t get_event(okmc_grid* g) {
  if (!g->free_events.empty()) {
    cudaEvent_t e = g->free_events.back();
    g->free_events.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void drain_profile(okmc_grid* g) {
  if (g->pending.empty()) return;
  cudaStreamSynchronize(g->st);
  for (auto& p : g->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    auto& slot = g->prof[p.name];
    slot.first += ms;
    slot.second += 1;
    g->free_events.push_back(p.a);
    g->free_events.push_back(p.b);
  }
  g->pending.clear();
}

// Launch wrapper: optional per-kernel CUDA events on the handle's stream.
template <class F>
int run(okmc_grid* g, const char* name, F f) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (g->profiling) {
    a = get_event(g);
    b = get_event(g);
    cudaEventRecord(a, g->st);
  }
  cudaError_t e = f();
  if (e != cudaSuccess) return cuda_fail(g, e, name);
  if (g->profiling) {
    cudaEventRecord(b, g->st);
    g->pending.push_back({name, a, b});
    if (g->pending.size() > 4096) drain_profile(g);
  }
  return OKMC_OK;
}

#define OKMC_TRY(x)              \
  do {                           \
    int _rc = (x);               \
    if (_rc != OKMC_OK) return _rc; \
  } while (0)

int3 dims(const okmc_grid* g) { return make_int3(g->n[0], g->n[1], g->n[2]); }
bool fp64(const okmc_grid* g) { return g->prec == OKMC_FP64_FIELDS; }
double quantum(const okmc_grid* g) { return fp64(g) ? std::ldexp(1.0, -40) : std::ldexp(1.0, -26); }
double qlimit(const okmc_grid* g) { return fp64(g) ? std::ldexp(1.0, 62) : 2147483647.0; }
size_t qsize(const okmc_grid* g) { return fp64(g) ? 8 : 4; }
size_t tsize(const okmc_grid* g) { return fp64(g) ? 8 : 4; }

// Tensor map of a fast-path spectrum (spec or spec2), or nullptr when the grid has none
const CUtensorMap* tmap(const okmc_grid* g, const void* spectrum) {
  if (!g->tm_ok) return nullptr;
  return spectrum == g->spec ? &g->tm_spec : spectrum == g->spec2 ? &g->tm_spec2 : nullptr;
}

// cuTensorMapEncodeTiled, reached through the runtime's driver entry point (no link
// against the driver library)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// A spectrum as the TMA pencil pass reads and writes it: 6 nz rows (comp * nz + kz) of
// 2 P floats, boxes of 16 floats by min(nz, 256) or nz / 2 rows, 64-byte swizzle
bool encode_spectrum_map(CUtensorMap* m, void* base, size_t P, int nz) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return false;
  const cuuint64_t dim[2] = {(cuuint64_t)(2 * P), (cuuint64_t)(6 * (size_t)nz)};
  const cuuint64_t stride[1] = {(cuuint64_t)(2 * P * sizeof(float))};
  const cuuint32_t box[2] = {16u, (cuuint32_t)(nz <= 256 ? nz : nz / 2)};
  const cuuint32_t estride[2] = {1u, 1u};
  if (nz > 256 && (nz % 2 != 0 || nz / 2 > 256)) return false;
  if (stride[0] % 16 != 0 || ((uintptr_t)base & 15) != 0) return false;
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dim, stride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int solve(okmc_grid* g) {
  if (g->sigma_valid) return OKMC_OK;
  PassCfg c = g->cfg;
  c.q = quantum(g);
  c.ncomp = 6;
  c.forward_only = 0;
  if (fp64(g)) {
    OKMC_TRY(run(g, "plane_fwd", [&] { return launch_plane_fwd<double, int64_t>((const int64_t*)g->eps, (C2<double>*)g->spec, c, g->st); }));
    OKMC_TRY(run(g, "pencil_green", [&] { return launch_pencil<double>((C2<double>*)g->spec, c, g->st); }));
    OKMC_TRY(run(g, "plane_inv", [&] { return launch_plane_inv<double>((const C2<double>*)g->spec, (double*)g->sig, c, g->st); }));
  } else if (g->fast) {
    // spec keeps the plane transforms of the eigenstrain between solves: only planes
    // whose eigenstrain changed are transformed again (bitwise the same result as a
    // full pass, since a clean plane's input is unchanged); the Green operator's
    // output goes to spec2
    c.dirty = g->d_dirty;
    OKMC_TRY(run(g, "plane_fwd", [&] { return launch_plane_fast(false, g->variant[0], g->eps, g->spec, c, g->st); }));
    c.dirty = nullptr;
    OKMC_TRY(run(g, "pencil_green", [&] { return launch_pencil_fast(g->variant[1], (const C2<float>*)g->spec, (C2<float>*)g->spec2, tmap(g, g->spec), tmap(g, g->spec2), c, g->st); }));
    OKMC_TRY(run(g, "plane_inv", [&] { return launch_plane_fast(true, g->variant[2], g->spec2, g->sig, c, g->st); }));
  } else {
    OKMC_TRY(run(g, "plane_fwd", [&] { return launch_plane_fwd<float, int32_t>((const int32_t*)g->eps, (C2<float>*)g->spec, c, g->st); }));
    OKMC_TRY(run(g, "pencil_green", [&] { return launch_pencil<float>((C2<float>*)g->spec, c, g->st); }));
    OKMC_TRY(run(g, "plane_inv", [&] { return launch_plane_inv<float>((const C2<float>*)g->spec, (float*)g->sig, c, g->st); }));
  }
  g->sigma_valid = true;
  g->solves += 1;
  return OKMC_OK;
}

int energies(okmc_grid* g, int want_cand, double kT = 0.0) {
  OKMC_TRY(solve(g));
  const double pref = -kKappa * g->h * g->h * g->h;
  RateArgs ra = {};
  if (kT > 0.0) {
    ra.rates = g->d_rates;
    ra.rsum = g->d_rsum;
    ra.negb = &g->d_state->negative_barriers;
    ra.nu0 = g->nu0;
    ra.kT = kT;
    ra.rkT = 1.0 / kT;
  }
  DilatedLists dl{};
  if (g->d_dl) {
    dl.ptr = g->d_dl;
    dl.end = g->d_dl + 2 * g->nd;
    dl.off = g->d_doff;
    dl.cnt = g->d_dcnt;
    dl.scnt = g->d_dscnt;
  }
  if (want_cand && g->nchunk > 0) {
    const ChunkArgs ca{g->d_cdef, g->d_c0, g->d_cpart, g->nchunk};
    OKMC_TRY(run(g, "energies", [&] {
      if (fp64(g))
        return launch_energy_chunks<double>((const double*)g->sig, dims(g), g->d_def, g->d_geo, g->nd, dl, ca, g->st);
      return launch_energy_chunks<float>((const float*)g->sig, dims(g), g->d_def, g->d_geo, g->nd, dl, ca, g->st);
    }));
    return run(g, "energies_finish", [&] {
      return launch_energy_finish(g->d_def, g->d_geo, g->nd, dl, ca, g->d_alpha, g->d_W, pref, g->d_E, g->d_Ec, ra, g->st);
    });
  }
  return run(g, "energies", [&] {
    if (fp64(g))
      return launch_energies<double>((const double*)g->sig, dims(g), g->d_def, g->d_geo, g->nd, g->d_ptr, g->d_off, g->d_cnt,
                                     g->d_alpha, g->d_W, pref, want_cand, g->d_order, g->nbig, g->d_E, g->d_Ec, ra, dl, g->st);
    return launch_energies<float>((const float*)g->sig, dims(g), g->d_def, g->d_geo, g->nd, g->d_ptr, g->d_off, g->d_cnt,
                                  g->d_alpha, g->d_W, pref, want_cand, g->d_order, g->nbig, g->d_E, g->d_Ec, ra, dl, g->st);
  });
}

int apply_moves(okmc_grid* g, int maxmoves) {
  return run(g, "apply_moves", [&] {
    if (fp64(g))
      return launch_apply_moves<int64_t>((int64_t*)g->eps, dims(g), g->d_geo, maxmoves, g->d_ptr, g->d_off, g->d_cnt,
                                         g->d_alpha, g->d_moves, g->d_state, 1.0 / quantum(g), qlimit(g), g->d_err, g->d_dirty, g->st);
    return launch_apply_moves<int32_t>((int32_t*)g->eps, dims(g), g->d_geo, maxmoves, g->d_ptr, g->d_off, g->d_cnt,
                                       g->d_alpha, g->d_moves, g->d_state, 1.0 / quantum(g), qlimit(g), g->d_err, g->d_dirty, g->st);
  });
}

int check_device_error(okmc_grid* g) {
  int e = 0;
  cudaError_t ce = cudaMemcpyAsync(&e, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(g->st);
  if (ce != cudaSuccess) return cuda_fail(g, ce, "device error check");
  if (e == 4) return fail(g, OKMC_ERANGE, "eigenstrain contribution outside the fixed-point range");
  if (e == 6) return fail(g, OKMC_ETIMEOUT, "a bounded wait for a bulk copy gave up");
  if (e) return fail(g, OKMC_ECUDA, "stencil construction inconsistency (code " + std::to_string(e) + ")");
  return OKMC_OK;
}

int copy_out(okmc_grid* g, void* dst, const void* src, size_t bytes, int on_device) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->st);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(g->st);
  if (e != cudaSuccess) return cuda_fail(g, e, "copy out");
  return OKMC_OK;
}

int validate_defects(okmc_grid* g, const okmc_defect* d, int nd) {
  const int nmin = std::min(g->n[0], std::min(g->n[1], g->n[2]));
  for (int i = 0; i < nd; ++i) {
    const okmc_defect& r = d[i];
    const std::string at = "defect " + std::to_string(i) + ": ";
    if (r.reserved != 0) return fail(g, OKMC_EINVAL, at + "reserved field must be 0");
    if (r.type < 0 || r.type > 2) return fail(g, OKMC_EINVAL, at + "unknown type");
    const int par = r.pos[0] & 1;
    for (int a = 0; a < 3; ++a) {
      if (r.pos[a] < 0 || r.pos[a] >= 2 * g->n[a]) return fail(g, OKMC_EINVAL, at + "position outside [0, 2n)");
      if ((r.pos[a] & 1) != par) return fail(g, OKMC_EINVAL, at + "position is not a bcc site");
    }
    if (!std::isfinite(r.Em_eV)) return fail(g, OKMC_EINVAL, at + "E_m not finite");
    if (r.mobility < 0 || r.mobility > 2) return fail(g, OKMC_EINVAL, at + "unknown mobility");
    int extent;
    if (r.type == OKMC_SIA_CLUSTER) {
      if (r.size < 1 || r.size > 1000000) return fail(g, OKMC_EINVAL, at + "cluster size out of range");
      if (r.axis < 0 || r.axis > 3) return fail(g, OKMC_EINVAL, at + "axis out of range");
      const double q = 3.0 * r.size / (8.0 * kPi);
      extent = (int)std::ceil(std::cbrt(q > 1.0 ? q : 1.0)) + 3;
    } else {
      if (!(r.radius_nm > 0.0) || !std::isfinite(r.radius_nm)) return fail(g, OKMC_EINVAL, at + "radius must be > 0");
      if (r.axis < 0 || r.axis > (r.type == OKMC_LOOP_111 ? 3 : 2)) return fail(g, OKMC_EINVAL, at + "axis out of range");
      extent = (int)std::ceil(r.radius_nm / g->h) + 2;
    }
    if (r.type == OKMC_LOOP_100 && r.mobility != OKMC_IMMOBILE)
      return fail(g, OKMC_EINVAL, at + "<100> loops are immobile");
    if (2 * extent + 1 > nmin) return fail(g, OKMC_EINVAL, at + "defect larger than half the grid");
  }
  return OKMC_OK;
}

// Self-term table W (translation invariant, so computed once per distinct shape):
// the scalar count fields of three defects' stencils (both classes) are transformed
// with the forward plane and pencil passes, and k_selfterm_partial sums them against
// the type tables Q_t, which k_qtable leaves in the (idle) stress buffer.
// want_W / want_D: which tables the shape batches sum (D, the dipole self parts, is
// built on first use by ensure_dipole_tables).
template <class T, class Q>
int build_self_terms(okmc_grid* g, bool want_W = true, bool want_D = false) {
  const size_t N = g->N;
  const int3 n = dims(g);
  const int nd = g->nd;
  std::vector<DefGeo> geo(nd);
  cudaError_t e = cudaMemcpyAsync(geo.data(), g->d_geo, nd * sizeof(DefGeo), cudaMemcpyDeviceToHost, g->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
  if (e != cudaSuccess) return cuda_fail(g, e, "geometry read back");
  // types: 1/2<111> axes 0-3, <100> axes 4-6, SIA cluster 7; e = s E_t
  QTypes qt{};
  int slot[8];
  for (int t = 0; t < 8; ++t) slot[t] = -1;
  std::vector<int> ty(nd);
  std::vector<double> s2(nd);
  for (int i = 0; i < nd; ++i) {
    const okmc_defect& r = g->h_def[i];
    const int t = r.type == OKMC_LOOP_111 ? r.axis : r.type == OKMC_LOOP_100 ? 4 + r.axis : 7;
    if (slot[t] < 0) {
      slot[t] = qt.nt++;
      double nrm = 0.0;
      for (int a = 0; a < 6; ++a) nrm = std::max(nrm, std::fabs(geo[i].e6[a]));
      for (int a = 0; a < 6; ++a) qt.e6[slot[t]][a] = geo[i].e6[a] / nrm;
    }
    const double* E = qt.e6[slot[t]];
    double num = 0.0, den = 0.0;
    for (int a = 0; a < 6; ++a) {
      num += geo[i].e6[a] * E[a];
      den += E[a] * E[a];
    }
    const double sc = num / den;
    for (int a = 0; a < 6; ++a)
      if (std::fabs(geo[i].e6[a] - sc * E[a]) > 1e-12 * std::fabs(sc))
        return fail(g, OKMC_ECUDA, "eigenstrain tensor not proportional to its type's");
    ty[i] = slot[t];
    s2[i] = sc * sc;
  }
  // one computation per distinct shape: loops by (type, axis, radius), clusters by size
  std::map<std::tuple<int, int, int64_t>, int> first;
  std::vector<int> rep(nd), reps;
  for (int i = 0; i < nd; ++i) {
    const okmc_defect& r = g->h_def[i];
    int64_t rb;
    std::memcpy(&rb, &r.radius_nm, sizeof(rb));
    const auto key = r.type == OKMC_SIA_CLUSTER ? std::make_tuple(r.type, 0, (int64_t)r.size) : std::make_tuple(r.type, r.axis, rb);
    auto it = first.find(key);
    if (it == first.end()) {
      first.emplace(key, i);
      rep[i] = i;
      reps.push_back(i);
    } else {
      rep[i] = it->second;
    }
  }
  T* qtab = (T*)g->sig;
  if ((size_t)qt.nt * g->P * g->n[2] > 6 * N) return fail(g, OKMC_EINVAL, "grid too small for the self-term tables");
  PassCfg c = g->cfg;
  c.q = 1.0;
  c.ncomp = 6;
  c.forward_only = 1;
  OKMC_TRY(run(g, "self_qtable", [&] { return launch_qtable<T>(qtab, c, qt, g->st); }));
  e = cudaMemsetAsync(g->eps, 0, 6 * N * sizeof(Q), g->st);
  if (e != cudaSuccess) return cuda_fail(g, e, "memset");
  const double pref = -kKappa * g->h * g->h * g->h / (double)N;
  const double2* phx = g->ph;
  const double2* phy = g->ph + (g->H + 1);
  const double2* phz = phy + g->n[1];
  for (size_t r0 = 0; r0 < reps.size(); r0 += 3) {
    WBatch b{};
    b.nb = (int)std::min<size_t>(3, reps.size() - r0);
    for (int d = 0; d < b.nb; ++d) {
      b.idx[d] = reps[r0 + d];
      b.type[d] = ty[b.idx[d]];
      b.s2[d] = s2[b.idx[d]];
    }
    OKMC_TRY(run(g, "self_fields", [&] { return launch_wfields<Q>((Q*)g->eps, n, g->d_ptr, g->d_off, g->d_cnt, b, g->st); }));
    if (g->fast) {
      OKMC_TRY(run(g, "plane_fwd", [&] { return launch_plane_fast(false, g->variant[0], g->eps, g->spec, c, g->st); }));
      OKMC_TRY(run(g, "pencil_fwd", [&] { return launch_pencil_fast(g->variant[1], (const C2<float>*)g->spec, (C2<float>*)g->spec, tmap(g, g->spec), tmap(g, g->spec), c, g->st); }));
    } else {
      OKMC_TRY(run(g, "plane_fwd", [&] { return launch_plane_fwd<T, Q>((const Q*)g->eps, (C2<T>*)g->spec, c, g->st); }));
      OKMC_TRY(run(g, "pencil_fwd", [&] { return launch_pencil<T>((C2<T>*)g->spec, c, g->st); }));
    }
    if (want_W)
      OKMC_TRY(run(g, "self_terms", [&] {
        return launch_selfterm<T>((const C2<T>*)g->spec, c, b, qtab, phx, phy, phz, g->d_partial, kSelfBlocks, g->d_alpha,
                                  pref, g->d_W, g->st);
      }));
    if (want_D)
      OKMC_TRY(run(g, "dipole_self", [&] {
        return launch_dipself<T, T>((const C2<T>*)g->spec, c, b, qtab, phx, phy, phz, g->d_partial, kSelfBlocks, g->d_alpha,
                                    g->d_geo, g->h * g->h * g->h / (double)N, g->d_D, g->st);
      }));
    e = cudaMemsetAsync(g->eps, 0, 6 * N * sizeof(Q), g->st);
    if (e != cudaSuccess) return cuda_fail(g, e, "memset");
  }
  if (reps.size() < (size_t)nd) {  // copy each shape's rows (W and D) to the defects that share it
    for (double* tab : {want_W ? g->d_W : nullptr, want_D ? g->d_D : nullptr}) {
      if (!tab) continue;
      std::vector<double> W((size_t)nd * 18);
      e = cudaMemcpyAsync(W.data(), tab, W.size() * sizeof(double), cudaMemcpyDeviceToHost, g->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
      for (int i = 0; i < nd && e == cudaSuccess; ++i)
        if (rep[i] != i) std::copy(W.begin() + (size_t)rep[i] * 18, W.begin() + (size_t)rep[i] * 18 + 18, W.begin() + (size_t)i * 18);
      if (e == cudaSuccess) e = cudaMemcpyAsync(tab, W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice, g->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
      if (e != cudaSuccess) return cuda_fail(g, e, "self-term copy");
    }
  }
  g->sigma_valid = false;
  return OKMC_OK;
}

// Dilated candidate lists of every (defect, class): sizes, offsets, fill.
// The energy lists (each voxel of the site and candidate stencils once, nine counts) of
// every defect and site class, and the chunk slots of the chunked energies over them
// (none when a defect has no list); work[i] receives the longer of defect i's two lists,
// or the site plus candidate stencil entries where a class has no list.
int build_dilated_lists(okmc_grid* g, const std::vector<int>& nnz, std::vector<int>& work) {
  const int nd = g->nd;
  int* d_n = nullptr;
  OKMC_TRY(dalloc(g, (void**)&d_n, 2 * nd * sizeof(int)));
  int rc = run(g, "dilate_count", [&] { return launch_dilate_count(g->d_geo, nd, g->d_ptr, g->d_off, g->d_cnt, d_n, g->st); });
  std::vector<int> cnt(2 * nd), se(4 * nd);
  cudaError_t e = cudaSuccess;
  if (rc == OKMC_OK) {
    e = cudaMemcpyAsync(cnt.data(), d_n, 2 * nd * sizeof(int), cudaMemcpyDeviceToHost, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
  }
  dfree(g, d_n);
  if (rc != OKMC_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(g, e, "dilated list sizes");
  long long tot = 0;
  for (int k = 0; k < 2 * nd; ++k) {
    se[k] = cnt[k] < 0 ? -1 : (int)tot;
    se[2 * nd + k] = cnt[k] < 0 ? -1 : (int)(tot + cnt[k]);
    if (cnt[k] > 0) tot += cnt[k];
  }
  if (tot > 0x7fffffffll) return fail(g, OKMC_ENOMEM, "too many dilated stencil entries");
  work.assign(nd, 0);
  for (int i = 0; i < nd; ++i)
    for (int c = 0; c < 2; ++c) {
      const int k = 2 * i + c;
      work[i] = std::max(work[i], cnt[k] >= 0 ? cnt[k] : nnz[k] + nnz[2 * i + 1 - c]);
    }
  OKMC_TRY(dalloc(g, (void**)&g->d_dl, 4 * nd * sizeof(int)));
  OKMC_TRY(dalloc(g, (void**)&g->d_doff, (size_t)tot * sizeof(int)));
  OKMC_TRY(dalloc(g, (void**)&g->d_dcnt, (size_t)tot * sizeof(unsigned long long)));
  OKMC_TRY(dalloc(g, (void**)&g->d_dscnt, (size_t)tot * sizeof(uint8_t)));
  e = cudaMemcpyAsync(g->d_dl, se.data(), se.size() * sizeof(int), cudaMemcpyHostToDevice, g->st);
  if (e != cudaSuccess) return cuda_fail(g, e, "dilated list offsets");
  DilatedLists dl{g->d_dl, g->d_dl + 2 * nd, g->d_doff, g->d_dcnt, g->d_dscnt};
  OKMC_TRY(run(g, "dilate_fill", [&] { return launch_dilate_fill(g->d_geo, nd, g->d_ptr, g->d_off, g->d_cnt, dl, g->d_err, g->st); }));
  OKMC_TRY(check_device_error(g));
  // chunk slots of the energies: ceil(max(len(i, 0), len(i, 1)) / kEnergyWarpEntries) per
  // defect, in defect order; none when any defect has no energy list
  g->nchunk = 0;
  bool lists = true;
  for (int k = 0; k < 2 * nd; ++k) lists = lists && cnt[k] >= 0;
  if (!lists) return OKMC_OK;
  std::vector<int> c0(nd), cdef;
  for (int i = 0; i < nd; ++i) {
    c0[i] = (int)cdef.size();
    const int len = std::max(cnt[2 * i], cnt[2 * i + 1]);
    for (int k = 0; k < (len + kEnergyWarpEntries - 1) / kEnergyWarpEntries; ++k) cdef.push_back(i);
  }
  if (cdef.empty()) return OKMC_OK;
  OKMC_TRY(dalloc(g, (void**)&g->d_cdef, cdef.size() * sizeof(int)));
  OKMC_TRY(dalloc(g, (void**)&g->d_c0, nd * sizeof(int)));
  OKMC_TRY(dalloc(g, (void**)&g->d_cpart, cdef.size() * 9 * sizeof(double)));
  e = cudaMemcpyAsync(g->d_cdef, cdef.data(), cdef.size() * sizeof(int), cudaMemcpyHostToDevice, g->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->d_c0, c0.data(), nd * sizeof(int), cudaMemcpyHostToDevice, g->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
  if (e != cudaSuccess) return cuda_fail(g, e, "energy chunks");
  g->nchunk = (int)cdef.size();
  return OKMC_OK;
}

int voxelise_all(okmc_grid* g) {
  // the defects' stencils are added to the dislocation lines' plastic strain, if any
  cudaError_t e = g->d_bg ? cudaMemcpyAsync(g->eps, g->d_bg, 6 * g->N * qsize(g), cudaMemcpyDeviceToDevice, g->st)
                          : cudaMemsetAsync(g->eps, 0, 6 * g->N * qsize(g), g->st);
  // every plane transform is stale (the self-term build also used spec as scratch)
  if (e == cudaSuccess) e = cudaMemsetAsync(g->d_dirty, 1, sizeof(int) * 6 * g->n[2], g->st);
  if (e != cudaSuccess) return cuda_fail(g, e, "memset");
  g->sigma_valid = false;
  return run(g, "voxelise", [&] {
    if (fp64(g))
      return launch_voxelise<int64_t>((int64_t*)g->eps, dims(g), g->d_def, g->d_geo, g->nd, g->d_ptr, g->d_off, g->d_cnt,
                                      g->d_alpha, 1.0 / quantum(g), qlimit(g), g->d_err, g->st);
    return launch_voxelise<int32_t>((int32_t*)g->eps, dims(g), g->d_def, g->d_geo, g->nd, g->d_ptr, g->d_off, g->d_cnt,
                                    g->d_alpha, 1.0 / quantum(g), qlimit(g), g->d_err, g->st);
  });
}

void free_defects(okmc_grid* g) {
  void** bufs[] = {(void**)&g->d_def, (void**)&g->d_geo, (void**)&g->d_ptr, (void**)&g->d_off, (void**)&g->d_cnt,
                   (void**)&g->d_alpha, (void**)&g->d_sumcnt, (void**)&g->d_nnz, (void**)&g->d_W, (void**)&g->d_D,
                   (void**)&g->d_dip, (void**)&g->d_E,
                   (void**)&g->d_Ec, (void**)&g->d_order, (void**)&g->d_rates, (void**)&g->d_rsum, (void**)&g->d_moves, (void**)&g->d_pos,
                   (void**)&g->d_dl, (void**)&g->d_doff, (void**)&g->d_dcnt, (void**)&g->d_dscnt,
                   (void**)&g->d_cdef, (void**)&g->d_c0, (void**)&g->d_cpart};
  for (void** b : bufs) {
    dfree(g, *b);
    *b = nullptr;
  }
  g->nd = 0;
  g->nbig = 0;
  g->nchunk = 0;
}

// Kernels of one step (solve, energies + rates, event, incremental field update)
// on g->st.  With capture set the solve is always included.
int step_body(okmc_grid* g, int mode, double kT, bool capture) {
  if (capture) g->sigma_valid = false;
  OKMC_TRY(energies(g, 1, kT));
  if (mode == OKMC_RESIDENCE) {
    OKMC_TRY(run(g, "event_residence", [&] {
      return launch_residence(g->d_def, g->nd, g->d_rates, g->d_rsum, dims(g), g->desc.seed, g->d_moves, g->d_state, g->st);
    }));
    OKMC_TRY(apply_moves(g, 1));
  } else {
    OKMC_TRY(run(g, "event_fixed_dt", [&] {
      return launch_fixed_dt(g->d_def, g->d_geo, g->nd, g->d_rates, g->nu0, kT, dims(g), g->desc.seed, g->d_moves,
                             g->d_state, g->st);
    }));
    OKMC_TRY(apply_moves(g, g->nd));
  }
  g->sigma_valid = false;
  return OKMC_OK;
}

void drop_graphs(okmc_grid* g) {
  for (auto& s : g->graphs) cudaGraphExecDestroy(s.exec);
  g->graphs.clear();
}

// Held while a step graph is captured and while device memory is allocated or freed
// by handle creation, defect setup and destruction, so that threads driving different
// handles (the request server's lanes) never allocate during another's capture.
std::recursive_mutex g_capture_mu;

// Capture one step of g into a graph on a private stream (the handle's stream may be
// the legacy stream, which cannot be captured); the graph is launched on g->st.
int capture_step(okmc_grid* g, int mode, double T, cudaGraphExec_t* out) {
  std::lock_guard<std::recursive_mutex> lk(g_capture_mu);
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(g, e, "capture stream");
  cudaStream_t keep = g->st;
  const bool prof = g->profiling;
  g->profiling = false;
  g->st = cs;
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  int rc = (e == cudaSuccess) ? step_body(g, mode, kBoltzmann * T, true) : cuda_fail(g, e, "begin capture");
  cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
  g->st = keep;
  g->profiling = prof;
  cudaStreamDestroy(cs);
  if (rc != OKMC_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e2 != cudaSuccess) return cuda_fail(g, e2, "end capture");
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(g, e, "graph instantiate");
  return OKMC_OK;
}

// Launch-variant autotuner of the fast passes: each variant that exists for the grid
// is timed on the grid's own buffers (one warm-up launch, then three launches
// between events) and the fastest is kept.  Every variant computes each line with
// the same arithmetic, so the choice changes the time and not the result.  Choices
// are cached per grid shape for the life of the process.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, std::array<int, 3>> g_tune_cache;  // shape -> variant of each pass

// The choices also persist across processes in a JSON file, one entry per device and
// grid shape: {"<device name>|<SMs>|<nx>x<ny>x<nz>|<schema>": [v0, v1, v2], ...}.  The file
// is $OKMC_TUNE_CACHE if set (set and empty: no file), else $XDG_CACHE_HOME/okmc/tune.json
// or ~/.cache/okmc/tune.json.  It is read once per process; after each new tuning it is
// rewritten with its current content merged in (a temporary file renamed over it, so a
// reader never sees half a file).  An unreadable or malformed file counts as empty.
constexpr const char* kTuneSchema = "passes-v3";  // bump when the variants of a pass change meaning
bool g_tune_file_read = false;
std::map<std::string, std::array<int, 3>> g_tune_file;

std::string tune_cache_path() {
  if (const char* p = std::getenv("OKMC_TUNE_CACHE")) return p;
  std::string dir;
  if (const char* x = std::getenv("XDG_CACHE_HOME")) dir = x;
  else if (const char* h = std::getenv("HOME")) dir = std::string(h) + "/.cache";
  else return "";
  return dir + "/okmc/tune.json";
}

std::map<std::string, std::array<int, 3>> parse_tune_file(const std::string& text) {
  std::map<std::string, std::array<int, 3>> out;
  size_t i = 0;
  while (true) {
    const size_t a = text.find('"', i);
    if (a == std::string::npos) break;
    const size_t b = text.find('"', a + 1);
    if (b == std::string::npos) return {};
    const std::string key = text.substr(a + 1, b - a - 1);
    const size_t l = text.find('[', b);
    const size_t r = text.find(']', b);
    if (l == std::string::npos || r == std::string::npos || r < l) return {};
    std::array<int, 3> v{};
    const char* q = text.c_str() + l + 1;
    for (int k = 0; k < 3; ++k) {
      char* end = nullptr;
      const long x = std::strtol(q, &end, 10);
      if (end == q || x < 0 || x > 30) return {};
      v[k] = (int)x;
      q = end;
      while (*q == ' ' || *q == ',' || *q == '\n' || *q == '\t') ++q;
    }
    out[key] = v;
    i = r + 1;
  }
  return out;
}

std::map<std::string, std::array<int, 3>> read_tune_file(const std::string& path) {
  std::FILE* f = path.empty() ? nullptr : std::fopen(path.c_str(), "rb");
  if (!f) return {};
  std::string text;
  char buf[4096];
  size_t k;
  while ((k = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, k);
  std::fclose(f);
  return parse_tune_file(text);
}

void write_tune_file(const std::string& path, const std::map<std::string, std::array<int, 3>>& m) {
  if (path.empty()) return;
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos)  // create the directory chain (errors surface at fopen)
    for (size_t p = path.find('/', 1); p != std::string::npos && p <= slash; p = path.find('/', p + 1))
      mkdir(path.substr(0, p).c_str(), 0755);
  const std::string tmp = path + ".tmp." + std::to_string((long long)getpid());
  std::FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return;
  std::fputs("{\n", f);
  size_t n = 0;
  for (const auto& kv : m)
    std::fprintf(f, "  \"%s\": [%d, %d, %d]%s\n", kv.first.c_str(), kv.second[0], kv.second[1], kv.second[2],
                 ++n < m.size() ? "," : "");
  std::fputs("}\n", f);
  const bool ok = std::fclose(f) == 0;
  if (!ok || std::rename(tmp.c_str(), path.c_str()) != 0) std::remove(tmp.c_str());
}

std::string tune_key(const okmc_grid* g) {
  int dev = 0;
  cudaDeviceProp prop{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "";
  std::string name = prop.name;
  for (char& ch : name)
    if (ch == '"' || ch == '|') ch = '_';
  return name + "|" + std::to_string(prop.multiProcessorCount) + "|" + std::to_string(g->n[0]) + "x" +
         std::to_string(g->n[1]) + "x" + std::to_string(g->n[2]) + "|" + kTuneSchema;
}

// One launch of each pass in the chosen variants on the zeroed spectra (and the zero
// field the grid starts with), so that the one-time launch setup of those kernels
// (attributes, the occupancy query behind the L2 prefetch distance) happens here and
// not inside a later step-graph capture.
int warm_passes(okmc_grid* g) {
  const size_t sbytes = 6 * g->n[2] * g->P * 2 * tsize(g);
  PassCfg c = g->cfg;
  c.dirty = nullptr;
  cudaError_t e = cudaMemsetAsync(g->spec, 0, sbytes, g->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->spec2, 0, sbytes, g->st);
  if (e == cudaSuccess) e = launch_plane_fast(false, g->variant[0], g->eps, g->spec, c, g->st);
  if (e == cudaSuccess)
    e = launch_pencil_fast(g->variant[1], (const C2<float>*)g->spec, (C2<float>*)g->spec2, tmap(g, g->spec), tmap(g, g->spec2), c, g->st);
  if (e == cudaSuccess) e = launch_plane_fast(true, g->variant[2], g->spec2, g->sig, c, g->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
  return e == cudaSuccess ? OKMC_OK : cuda_fail(g, e, "warm-up launches");
}

int autotune(okmc_grid* g) {
  if (!g->fast) return OKMC_OK;
  // OKMC_VARIANTS=a,b,c pins the variant of each pass (where it exists) without timing,
  // e.g. under a profiler; OKMC_TUNE=0 keeps variant 0 of every pass
  if (const char* pin = std::getenv("OKMC_VARIANTS")) {
    int v[3] = {0, 0, 0};
    if (std::sscanf(pin, "%d,%d,%d", &v[0], &v[1], &v[2]) == 3)
      for (int p = 0; p < 3; ++p)
        if (v[p] >= 0 && v[p] < 31 && ((g->avail[p] >> v[p]) & 1)) g->variant[p] = v[p];
    return warm_passes(g);
  }
  const char* env = std::getenv("OKMC_TUNE");
  if (env && env[0] == '0') return warm_passes(g);
  const auto key = std::make_tuple(g->n[0], g->n[1], g->n[2]);
  const std::string fkey = tune_key(g);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      for (int p = 0; p < 3; ++p) g->variant[p] = it->second[p];
      return OKMC_OK;
    }
    if (!g_tune_file_read) {
      g_tune_file = read_tune_file(tune_cache_path());
      g_tune_file_read = true;
    }
    auto ft = fkey.empty() ? g_tune_file.end() : g_tune_file.find(fkey);
    if (ft != g_tune_file.end()) {
      bool ok = true;
      for (int p = 0; p < 3; ++p) ok = ok && ((g->avail[p] >> ft->second[p]) & 1);
      if (ok) {
        for (int p = 0; p < 3; ++p) g->variant[p] = ft->second[p];
        g_tune_cache[key] = ft->second;
        return warm_passes(g);  // first grid of this shape in the process: one-time launch set-up
      }
    }
  }
  const size_t sbytes = 6 * g->n[2] * g->P * 2 * tsize(g);
  cudaError_t e = cudaMemsetAsync(g->spec, 0, sbytes, g->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->spec2, 0, sbytes, g->st);
  if (e != cudaSuccess) return cuda_fail(g, e, "tune");
  PassCfg c = g->cfg;
  c.dirty = nullptr;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return cuda_fail(g, cudaGetLastError(), "tune event");
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return cuda_fail(g, cudaGetLastError(), "tune event");
  }
  // three interleaved rounds, the best of each variant, and variant 0 kept unless
  // another is more than 2% faster (robust against a noisy or shared device)
  // (the forward pass runs on every plane here, and on the zero field the grid starts
  // with, so the plane transforms it leaves in spec stay those of the field); a pass
  // with a single variant is not timed
  for (int pass = 0; pass <= 2 && e == cudaSuccess; ++pass) {
    if (g->avail[pass] == 1) continue;
    auto launch = [&](int v) {
      if (pass == 0) return launch_plane_fast(false, v, g->eps, g->spec, c, g->st);
      return pass == 1 ? launch_pencil_fast(v, (const C2<float>*)g->spec, (C2<float>*)g->spec2, tmap(g, g->spec), tmap(g, g->spec2), c, g->st)
                       : launch_plane_fast(true, v, g->spec2, g->sig, c, g->st);
    };
    float best[16];
    for (int v = 0; v < 16; ++v) best[v] = 1e30f;
    for (int round = 0; round < 3 && e == cudaSuccess; ++round) {
      for (int v = 0; v < 16 && e == cudaSuccess; ++v) {
        if (!((g->avail[pass] >> v) & 1)) continue;
        e = launch(v);
        if (e == cudaSuccess) e = cudaEventRecord(a, g->st);
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = launch(v);
        if (e == cudaSuccess) e = cudaEventRecord(b, g->st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess) best[v] = std::min(best[v], ms);
      }
    }
    int pick = 0;
    for (int v = 1; v < 16; ++v)
      if (best[v] < 0.98f * best[0] && best[v] < best[pick]) pick = v;
    g->variant[pass] = pick;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(g, e, "tune");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = {g->variant[0], g->variant[1], g->variant[2]};
  if (!fkey.empty()) {
    const std::string path = tune_cache_path();
    auto merged = read_tune_file(path);
    merged[fkey] = g_tune_cache[key];
    write_tune_file(path, merged);
    g_tune_file = merged;
  }
  return OKMC_OK;
}

// The dipole self parts D, summed on first use (a dipole-free run pays nothing for
// them).  The shape batches use the field buffers as scratch, so the eigenstrain field
// is voxelised again from the current positions after them.
int ensure_dipole_tables(okmc_grid* g) {
  if (g->dip_valid) return OKMC_OK;
  std::lock_guard<std::recursive_mutex> lk(g_capture_mu);  // as set_defects: setup work
  OKMC_TRY((fp64(g) ? build_self_terms<double, int64_t>(g, false, true) : build_self_terms<float, int32_t>(g, false, true)));
  OKMC_TRY(voxelise_all(g));
  OKMC_TRY(check_device_error(g));
  g->dip_valid = true;
  return OKMC_OK;
}

}  // namespace

// ================================================================== C ABI
extern "C" {

const char* okmc_last_error(const okmc_grid* g) {
  if (!g) return "null handle";
  return g->err.c_str();
}

int okmc_grid_create(const okmc_grid_desc* d, okmc_grid** out) {
  std::lock_guard<std::recursive_mutex> lk(g_capture_mu);
  if (!d || !out) return OKMC_EINVAL;
  *out = nullptr;
  for (int a = 0; a < 3; ++a)
    if (!factor_ok(d->n[a])) return OKMC_EINVAL;
  if (!(d->voxel_nm > 0.0) || !std::isfinite(d->voxel_nm)) return OKMC_EINVAL;
  if (!std::isfinite(d->C11) || !std::isfinite(d->C12) || !std::isfinite(d->C44)) return OKMC_EINVAL;
  if (!(d->C11 - d->C12 > 0.0) || !(d->C11 + 2.0 * d->C12 > 0.0) || !(d->C44 > 0.0)) return OKMC_EINVAL;
  if (d->k0_mode != OKMC_MEAN_STRESS_ZERO && d->k0_mode != OKMC_MEAN_STRAIN_ZERO) return OKMC_EINVAL;
  if (d->precision != OKMC_FP32_FIELDS && d->precision != OKMC_FP64_FIELDS) return OKMC_EINVAL;
  if (d->nu0 < 0.0 || !std::isfinite(d->nu0)) return OKMC_EINVAL;
  okmc_grid* g = new (std::nothrow) okmc_grid();
  if (!g) return OKMC_ENOMEM;
  g->desc = *d;
  for (int a = 0; a < 3; ++a) g->n[a] = d->n[a];
  g->H = g->n[0] / 2;
  g->N = (size_t)g->n[0] * g->n[1] * g->n[2];
  g->P = (size_t)(g->H + 1) * g->n[1];
  g->h = d->voxel_nm;
  g->nu0 = d->nu0 > 0.0 ? d->nu0 : 1e13;
  g->prec = d->precision;
  g->st = (cudaStream_t)d->stream;
  const bool f64 = fp64(g);
  const int cs = f64 ? pick_cluster<double>(g->H, g->n[1], kSmemLimit) : pick_cluster<float>(g->H, g->n[1], kSmemLimit);
  const int tw = f64 ? pick_tile<double>(g->n[1], g->n[2], kSmemLimit) : pick_tile<float>(g->n[1], g->n[2], kSmemLimit);
  if (!cs || !tw) {
    delete g;
    return OKMC_EINVAL;
  }
  int rc = OKMC_OK;
  auto cleanup = [&](int code) {
    okmc_grid_destroy(g);
    return code;
  };
  if ((rc = dalloc(g, &g->eps, 6 * g->N * qsize(g)))) return cleanup(rc);
  if ((rc = dalloc(g, &g->sig, 6 * g->N * tsize(g)))) return cleanup(rc);
  if ((rc = dalloc(g, &g->spec, 6 * g->n[2] * g->P * 2 * tsize(g)))) return cleanup(rc);
  if ((rc = dalloc(g, (void**)&g->d_state, sizeof(DevState)))) return cleanup(rc);
  if ((rc = dalloc(g, (void**)&g->d_err, sizeof(int)))) return cleanup(rc);
  if ((rc = dalloc(g, (void**)&g->d_partial, sizeof(double) * 30 * kSelfBlocks))) return cleanup(rc);
  // twiddle tables: w_H^k, w_ny^k, w_nz^k, exp(-2 pi i k/nx) for k <= H
  size_t off_tw[4], off_lw[4] = {0, 0, 0, 0};
  cudaError_t e;
  if (f64) {
    std::vector<C2<double>> t;
    off_tw[0] = t.size(); twiddles(t, g->H, g->H, -1.0);
    off_tw[1] = t.size(); twiddles(t, g->n[1], g->n[1], -1.0);
    off_tw[2] = t.size(); twiddles(t, g->n[2], g->n[2], -1.0);
    off_tw[3] = t.size(); twiddles(t, g->n[0], g->H + 1, -1.0);
    if ((rc = dalloc(g, &g->tw, t.size() * sizeof(t[0])))) return cleanup(rc);
    // on the handle's stream (which may be non-blocking, so unordered with the legacy
    // stream), then waited for: the host table must outlive the copy
    e = cudaMemcpyAsync(g->tw, t.data(), t.size() * sizeof(t[0]), cudaMemcpyHostToDevice, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    for (int k = 0; k < 4; ++k) off_tw[k] *= sizeof(C2<double>);
  } else {
    std::vector<C2<float>> t;
    off_tw[0] = t.size(); twiddles(t, g->H, g->H, -1.0);
    off_tw[1] = t.size(); twiddles(t, g->n[1], g->n[1], -1.0);
    off_tw[2] = t.size(); twiddles(t, g->n[2], g->n[2], -1.0);
    off_tw[3] = t.size(); twiddles(t, g->n[0], g->H + 1, -1.0);
    if ((rc = dalloc(g, &g->tw, t.size() * sizeof(t[0])))) return cleanup(rc);
    // on the handle's stream (which may be non-blocking, so unordered with the legacy
    // stream), then waited for: the host table must outlive the copy
    e = cudaMemcpyAsync(g->tw, t.data(), t.size() * sizeof(t[0]), cudaMemcpyHostToDevice, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    for (int k = 0; k < 4; ++k) off_tw[k] *= sizeof(C2<float>);
    if (e == cudaSuccess) {
      std::vector<C2<float>> l;
      off_lw[0] = l.size(); balanced_twiddles(l, g->H, g->H, twiddle_use(g->H));
      off_lw[1] = l.size(); balanced_twiddles(l, g->n[1], g->n[1], twiddle_use(g->n[1]));
      off_lw[2] = l.size(); balanced_twiddles(l, g->n[2], g->n[2], twiddle_use(g->n[2]));
      off_lw[3] = l.size(); balanced_twiddles(l, g->n[0], g->H + 1, {});
      if ((rc = dalloc(g, &g->ftw, l.size() * sizeof(l[0])))) return cleanup(rc);
      e = cudaMemcpyAsync(g->ftw, l.data(), l.size() * sizeof(l[0]), cudaMemcpyHostToDevice, g->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
      for (int k = 0; k < 4; ++k) off_lw[k] *= sizeof(l[0]);
    }
  }
  if (e != cudaSuccess) return cleanup(OKMC_ECUDA);
  // phase tables exp(+2 pi i f / n) for the self-term shifts (f: signed frequency)
  {
    std::vector<double2> ph;
    auto add = [&](int nn, int count, int half) {
      for (int k = 0; k < count; ++k) {
        const int f = (half ? (k < nn / 2 ? k : k - nn) : (k < nn / 2 ? k : k - nn));
        const double ang = 2.0 * kPi * (double)f / (double)nn;
        ph.push_back(make_double2(std::cos(ang), std::sin(ang)));
      }
    };
    add(g->n[0], g->H + 1, 1);
    add(g->n[1], g->n[1], 0);
    add(g->n[2], g->n[2], 0);
    if ((rc = dalloc(g, (void**)&g->ph, ph.size() * sizeof(double2)))) return cleanup(rc);
    e = cudaMemcpyAsync(g->ph, ph.data(), ph.size() * sizeof(double2), cudaMemcpyHostToDevice, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    if (e != cudaSuccess) return cleanup(OKMC_ECUDA);
  }
  PassCfg& c = g->cfg;
  c.nx = g->n[0];
  c.ny = g->n[1];
  c.nz = g->n[2];
  c.H = g->H;
  c.ncomp = 6;
  c.cs = cs;
  c.tw_w = tw;
  c.k0_mode = d->k0_mode;
  c.forward_only = 0;
  c.q = quantum(g);
  c.C11 = d->C11;
  c.C12 = d->C12;
  c.C44 = d->C44;
  {
    const double rN = 1.0 / ((double)c.nx * c.ny * c.nz);
    const double Cd[3] = {c.C11, c.C12, c.C44};
    for (int a = 0; a < 3; ++a) {
      c.fC[a] = (float)Cd[a];
      c.fCs[a] = (float)(Cd[a] * rN);
    }
  }
  for (int a = 0; a < 3; ++a) c.rn[a] = (float)(1.0 / g->n[a]);
  c.pH = make_plan(g->H);
  c.pY = make_plan(g->n[1]);
  c.pZ = make_plan(g->n[2]);
  c.twH = (const char*)g->tw + off_tw[0];
  c.twY = (const char*)g->tw + off_tw[1];
  c.twZ = (const char*)g->tw + off_tw[2];
  c.untw = (const char*)g->tw + off_tw[3];
  if (g->ftw) {
    c.ftwH = (const char*)g->ftw + off_lw[0];
    c.ftwY = (const char*)g->ftw + off_lw[1];
    c.ftwZ = (const char*)g->ftw + off_lw[2];
    c.ftwU = (const char*)g->ftw + off_lw[3];
  }
  c.err = g->d_err;
  // OKMC_GENERIC_FFT=1 keeps the generic passes (diagnostics and cross-checks)
  {
    const char* env = std::getenv("OKMC_GENERIC_FFT");
    g->fast = !f64 && fast_solve_supported(c) && !(env && env[0] == '1');
  }
  if (g->fast && (rc = dalloc(g, &g->spec2, 6 * g->n[2] * g->P * 2 * tsize(g)))) return cleanup(rc);
  if (g->fast) {
    g->tm_ok = encode_spectrum_map(&g->tm_spec, g->spec, g->P, g->n[2]) &&
               encode_spectrum_map(&g->tm_spec2, g->spec2, g->P, g->n[2]);
    g->avail[1] = pencil_variant_mask(c) & (g->tm_ok ? ~0 : ~4);  // variant 2 stages by TMA
    g->avail[0] = plane_fwd_variant_mask(c);
    g->avail[2] = plane_inv_variant_mask(c);
  }
  if ((rc = dalloc(g, (void**)&g->d_dirty, sizeof(int) * 6 * g->n[2]))) return cleanup(rc);
  if (cudaMemsetAsync(g->d_dirty, 1, sizeof(int) * 6 * g->n[2], g->st) != cudaSuccess) return cleanup(OKMC_ECUDA);
  if (cudaMemsetAsync(g->eps, 0, 6 * g->N * qsize(g), g->st) != cudaSuccess) return cleanup(OKMC_ECUDA);
  if (cudaMemsetAsync(g->d_state, 0, sizeof(DevState), g->st) != cudaSuccess) return cleanup(OKMC_ECUDA);
  if (cudaMemsetAsync(g->d_err, 0, sizeof(int), g->st) != cudaSuccess) return cleanup(OKMC_ECUDA);
  if (cudaStreamSynchronize(g->st) != cudaSuccess) return cleanup(OKMC_ECUDA);
  if ((rc = autotune(g))) return cleanup(rc);
  // OKMC_TMA_EXTRA_TX=b (a test hook, taken after the tuner's launches): the TMA-staged
  // pencil pass expects b bytes beyond its copies, so that its bounded wait runs out
  if (const char* x = std::getenv("OKMC_TMA_EXTRA_TX")) c.tx_extra = std::max(0, std::min(atoi(x), 1 << 16));
  *out = g;
  return OKMC_OK;
}

int okmc_isotropic_stiffness(double mu_GPa, double nu, double C[3]) {
  if (!C || !(mu_GPa > 0.0) || !std::isfinite(mu_GPa) || !(nu > -1.0) || !(nu < 0.5)) return OKMC_EINVAL;
  const double lam = 2.0 * mu_GPa * nu / (1.0 - 2.0 * nu);
  C[0] = lam + 2.0 * mu_GPa;
  C[1] = lam;
  C[2] = mu_GPa;
  return OKMC_OK;
}

size_t okmc_estimate_field_bytes(const okmc_grid_desc* d) {
  if (!d || d->n[0] < 1 || d->n[1] < 1 || d->n[2] < 1) return 0;
  const bool f64 = d->precision == OKMC_FP64_FIELDS;
  const size_t N = (size_t)d->n[0] * d->n[1] * d->n[2];
  const size_t H = d->n[0] / 2, P = (H + 1) * d->n[1], w = f64 ? 8 : 4;
  PassCfg c{};
  c.nx = d->n[0];
  c.ny = d->n[1];
  c.nz = d->n[2];
  c.ncomp = 6;
  const char* env = std::getenv("OKMC_GENERIC_FFT");
  const bool fast = !f64 && fast_solve_supported(c) && !(env && env[0] == '1');
  size_t b = 6 * N * w * 2 + 6 * d->n[2] * P * 2 * w * (fast ? 2 : 1);
  b += sizeof(DevState) + sizeof(int) + sizeof(double) * 30 * kSelfBlocks + sizeof(int) * 6 * d->n[2];
  b += (2 * H + 1 + d->n[1] + d->n[2]) * 2 * w + (H + 1 + d->n[1] + d->n[2]) * sizeof(double2);
  if (!f64) b += (2 * H + 1 + d->n[1] + d->n[2]) * 2 * w;
  return b;
}

int okmc_grid_destroy(okmc_grid* g) {
  if (!g) return OKMC_OK;
  std::lock_guard<std::recursive_mutex> lk(g_capture_mu);
  cudaStreamSynchronize(g->st);
  for (auto& p : g->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto ev : g->free_events) cudaEventDestroy(ev);
  drop_graphs(g);
  for (auto& a : g->allocs) cudaFree(a.first);
  delete g;
  return OKMC_OK;
}

int okmc_set_stream(okmc_grid* g, void* stream) {
  if (!g) return OKMC_EINVAL;
  drain_profile(g);
  cudaStreamSynchronize(g->st);
  g->st = (cudaStream_t)stream;
  return OKMC_OK;
}

int okmc_set_defects(okmc_grid* g, const okmc_defect* defs, int32_t nd) {
  if (!g) return OKMC_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(g_capture_mu);
  if (nd < 0 || (nd > 0 && !defs)) return fail(g, OKMC_EINVAL, "bad defect array");
  try {
    OKMC_TRY(validate_defects(g, defs, nd));
    cudaStreamSynchronize(g->st);
    drop_graphs(g);
    g->gen += 1;
    free_defects(g);
    g->h_def.assign(defs, defs + nd);
    g->nd = nd;
    g->any_mobile = false;
    for (int i = 0; i < nd; ++i) g->any_mobile |= defs[i].mobility != OKMC_IMMOBILE;
    const size_t n1 = nd > 0 ? nd : 1;
    OKMC_TRY(dalloc(g, (void**)&g->d_def, n1 * sizeof(okmc_defect)));
    OKMC_TRY(dalloc(g, (void**)&g->d_geo, n1 * sizeof(DefGeo)));
    OKMC_TRY(dalloc(g, (void**)&g->d_ptr, (2 * n1 + 1) * sizeof(int)));
    OKMC_TRY(dalloc(g, (void**)&g->d_alpha, 2 * n1 * sizeof(double)));
    OKMC_TRY(dalloc(g, (void**)&g->d_sumcnt, 2 * n1 * sizeof(long long)));
    OKMC_TRY(dalloc(g, (void**)&g->d_nnz, 2 * n1 * sizeof(int)));
    OKMC_TRY(dalloc(g, (void**)&g->d_W, 18 * n1 * sizeof(double)));
    OKMC_TRY(dalloc(g, (void**)&g->d_D, 18 * n1 * sizeof(double)));
    OKMC_TRY(dalloc(g, (void**)&g->d_dip, 9 * n1 * sizeof(double)));
    OKMC_TRY(dalloc(g, (void**)&g->d_E, n1 * sizeof(double)));
    OKMC_TRY(dalloc(g, (void**)&g->d_Ec, 8 * n1 * sizeof(double)));
    OKMC_TRY(dalloc(g, (void**)&g->d_rates, 8 * n1 * sizeof(double)));
    OKMC_TRY(dalloc(g, (void**)&g->d_order, n1 * sizeof(int)));
    OKMC_TRY(dalloc(g, (void**)&g->d_rsum, n1 * sizeof(double)));
    OKMC_TRY(dalloc(g, (void**)&g->d_moves, n1 * sizeof(Move)));
    OKMC_TRY(dalloc(g, (void**)&g->d_pos, 3 * n1 * sizeof(int)));
    cudaError_t e = cudaSuccess;
    if (nd) e = cudaMemcpyAsync(g->d_def, defs, nd * sizeof(okmc_defect), cudaMemcpyHostToDevice, g->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_err, 0, sizeof(int), g->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_state, 0, sizeof(DevState), g->st);
    if (e != cudaSuccess) return cuda_fail(g, e, "upload");
    g->solves = 0;
    std::vector<int> ptr(2 * n1 + 1, 0), nnz;
    if (nd) {
      OKMC_TRY(run(g, "defect_setup", [&] { return launch_defect_setup(g->d_def, g->d_geo, nd, g->h, g->st); }));
      OKMC_TRY(run(g, "stencil_count", [&] { return launch_stencil_count(g->d_geo, nd, g->d_nnz, g->d_sumcnt, g->st); }));
      nnz.resize(2 * nd);
      e = cudaMemcpyAsync(nnz.data(), g->d_nnz, 2 * nd * sizeof(int), cudaMemcpyDeviceToHost, g->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
      if (e != cudaSuccess) return cuda_fail(g, e, "stencil sizes");
      long long tot = 0;
      for (int k = 0; k < 2 * nd; ++k) {
        ptr[k] = (int)tot;
        tot += nnz[k];
      }
      ptr[2 * nd] = (int)tot;
      if (tot > 0x7fffffffll) return fail(g, OKMC_ENOMEM, "too many stencil entries");
      OKMC_TRY(dalloc(g, (void**)&g->d_off, (size_t)tot * sizeof(int)));
      OKMC_TRY(dalloc(g, (void**)&g->d_cnt, (size_t)tot));
    } else {
      OKMC_TRY(dalloc(g, (void**)&g->d_off, 16));
      OKMC_TRY(dalloc(g, (void**)&g->d_cnt, 16));
    }
    e = cudaMemcpyAsync(g->d_ptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice, g->st);
    if (e != cudaSuccess) return cuda_fail(g, e, "stencil offsets");
    if (nd) {
      OKMC_TRY(run(g, "stencil_fill", [&] {
        return launch_stencil_fill(g->d_geo, nd, g->d_ptr, g->d_sumcnt, g->d_off, g->d_cnt, g->d_alpha, g->d_err, g->st);
      }));
      OKMC_TRY(check_device_error(g));
      std::vector<int> work;
      OKMC_TRY(build_dilated_lists(g, nnz, work));
      // energies order: longest energy list first; the nbig lists longer than one pass of
      // a warp take a block each, the rest one warp each
      std::vector<int> order(nd);
      for (int i = 0; i < nd; ++i) order[i] = i;
      std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
      g->nbig = 0;
      while (g->nbig < nd && work[order[g->nbig]] > kEnergyWarpEntries) ++g->nbig;
      e = cudaMemcpyAsync(g->d_order, order.data(), nd * sizeof(int), cudaMemcpyHostToDevice, g->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
      if (e != cudaSuccess) return cuda_fail(g, e, "energy order");
      OKMC_TRY((fp64(g) ? build_self_terms<double, int64_t>(g) : build_self_terms<float, int32_t>(g)));
    }
    g->dip_valid = false;
    OKMC_TRY(voxelise_all(g));
    OKMC_TRY(check_device_error(g));
    g->sigma_valid = false;
    return OKMC_OK;
  } catch (const std::bad_alloc&) {
    return fail(g, OKMC_ENOMEM, "host allocation failed");
  }
}

int okmc_get_defects(okmc_grid* g, okmc_defect* out, int32_t n) {
  if (!g || (n > 0 && !out)) return OKMC_EINVAL;
  if (n != g->nd) return fail(g, OKMC_EINVAL, "count differs from the defect set");
  if (!n) return OKMC_OK;
  return copy_out(g, out, g->d_def, n * sizeof(okmc_defect), 0);
}

int okmc_set_positions(okmc_grid* g, const int32_t* pos, int32_t n, int on_device) {
  if (!g || (n > 0 && !pos)) return OKMC_EINVAL;
  if (n != g->nd) return fail(g, OKMC_EINVAL, "count differs from the defect set");
  if (!n) return OKMC_OK;
  if (!on_device) {
    for (int i = 0; i < n; ++i) {
      const int par = pos[3 * i] & 1;
      for (int a = 0; a < 3; ++a) {
        if (pos[3 * i + a] < 0 || pos[3 * i + a] >= 2 * g->n[a]) return fail(g, OKMC_EINVAL, "position outside [0, 2n)");
        if ((pos[3 * i + a] & 1) != par) return fail(g, OKMC_EINVAL, "position is not a bcc site");
      }
    }
  }
  cudaError_t e = cudaMemcpyAsync(g->d_pos, pos, 3 * n * sizeof(int), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(&g->d_state->nmoves, 0, sizeof(int), g->st);
  if (e != cudaSuccess) return cuda_fail(g, e, "positions upload");
  OKMC_TRY(run(g, "diff_positions", [&] { return launch_diff_positions(g->d_def, g->d_pos, n, g->d_moves, g->d_state, g->st); }));
  OKMC_TRY(apply_moves(g, n));
  g->sigma_valid = false;
  return OKMC_OK;
}

int okmc_get_positions(okmc_grid* g, int32_t* pos, int32_t n, int on_device) {
  if (!g || (n > 0 && !pos)) return OKMC_EINVAL;
  if (n != g->nd) return fail(g, OKMC_EINVAL, "count differs from the defect set");
  if (!n) return OKMC_OK;
  OKMC_TRY(run(g, "gather_positions", [&] { return launch_gather_positions(g->d_def, g->d_pos, n, g->st); }));
  return copy_out(g, pos, g->d_pos, 3 * n * sizeof(int), on_device);
}

int okmc_solve_stress(okmc_grid* g, void* sigma_out, int out_on_device) {
  if (!g) return OKMC_EINVAL;
  OKMC_TRY(solve(g));
  if (!sigma_out) return OKMC_OK;
  OKMC_TRY(copy_out(g, sigma_out, g->sig, 6 * g->N * tsize(g), out_on_device));
  return out_on_device ? OKMC_OK : check_device_error(g);  // the copy synchronised the stream already
}

int okmc_eigenstrain(okmc_grid* g, void* eps_out, int out_on_device) {
  if (!g || !eps_out) return OKMC_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(g_capture_mu);  // allocates: not during another thread's capture
  void* tmp = nullptr;
  OKMC_TRY(dalloc(g, &tmp, 6 * g->N * tsize(g)));
  int rc = run(g, "fixed_to_real", [&] {
    if (fp64(g)) return launch_fixed_to_real<int64_t, double>((const int64_t*)g->eps, (double*)tmp, 6 * g->N, quantum(g), g->st);
    return launch_fixed_to_real<int32_t, float>((const int32_t*)g->eps, (float*)tmp, 6 * g->N, quantum(g), g->st);
  });
  if (rc == OKMC_OK) rc = copy_out(g, eps_out, tmp, 6 * g->N * tsize(g), out_on_device);
  cudaStreamSynchronize(g->st);
  dfree(g, tmp);
  return rc;
}

int okmc_interaction_energies(okmc_grid* g, double* E, int out_on_device) {
  if (!g || !E) return OKMC_EINVAL;
  if (!g->nd) return OKMC_OK;
  OKMC_TRY(energies(g, 0));
  return copy_out(g, E, g->d_E, g->nd * sizeof(double), out_on_device);
}

int okmc_candidate_energies(okmc_grid* g, double* E, uint8_t* valid, int out_on_device) {
  if (!g || !E) return OKMC_EINVAL;
  if (!g->nd) return OKMC_OK;
  OKMC_TRY(energies(g, 1));
  OKMC_TRY(copy_out(g, E, g->d_Ec, g->nd * 8 * sizeof(double), out_on_device));
  if (valid) {
    std::vector<uint8_t> v(8 * g->nd, 0);
    for (int i = 0; i < g->nd; ++i) {
      const okmc_defect& r = g->h_def[i];
      int mask = 0;
      if (r.mobility == OKMC_THREE_D) mask = 0xFF;
      if (r.mobility == OKMC_ONE_D) {
        const int jp = 4 * (r.axis != 1) + 2 * (r.axis != 2) + (r.axis != 3);
        mask = (1 << jp) | (1 << (7 - jp));
      }
      for (int j = 0; j < 8; ++j) v[8 * i + j] = (mask >> j) & 1;
    }
    cudaError_t e = cudaMemcpyAsync(valid, v.data(), v.size(), out_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    if (e != cudaSuccess) return cuda_fail(g, e, "valid mask");
  }
  return OKMC_OK;
}

int okmc_dipole_energies(okmc_grid* g, double* E, double* Ec, int out_on_device) {
  if (!g || !E) return OKMC_EINVAL;
  if (!g->nd) return OKMC_OK;
  OKMC_TRY(ensure_dipole_tables(g));
  OKMC_TRY(solve(g));
  const double h3 = g->h * g->h * g->h;
  OKMC_TRY(run(g, "dipole_energies", [&] {
    if (fp64(g))
      return launch_dipole_energies<double>((const double*)g->sig, dims(g), g->d_def, g->d_geo, g->d_D, g->nd, h3, g->d_dip,
                                            g->d_dip + g->nd, g->st);
    return launch_dipole_energies<float>((const float*)g->sig, dims(g), g->d_def, g->d_geo, g->d_D, g->nd, h3, g->d_dip,
                                         g->d_dip + g->nd, g->st);
  }));
  OKMC_TRY(copy_out(g, E, g->d_dip, g->nd * sizeof(double), out_on_device));
  if (Ec) OKMC_TRY(copy_out(g, Ec, g->d_dip + g->nd, g->nd * 8 * sizeof(double), out_on_device));
  return OKMC_OK;
}

int okmc_dipole_self_terms(okmc_grid* g, double* D, int out_on_device) {
  if (!g || !D) return OKMC_EINVAL;
  if (!g->nd) return OKMC_OK;
  OKMC_TRY(ensure_dipole_tables(g));
  return copy_out(g, D, g->d_D, g->nd * 18 * sizeof(double), out_on_device);
}

int okmc_set_dislocations(okmc_grid* g, const double* points, const int32_t* counts, const int32_t* closed,
                          const double* burgers, int32_t n_lines, double ds_max_nm) {
  if (!g) return OKMC_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(g_capture_mu);
  if (n_lines < 0 || (n_lines > 0 && (!points || !counts || !closed || !burgers)))
    return fail(g, OKMC_EINVAL, "bad dislocation arrays");
  if (!(ds_max_nm <= 0.0) && !(ds_max_nm > 0.0 && std::isfinite(ds_max_nm))) return fail(g, OKMC_EINVAL, "bad ds_max_nm");
  const double ds = ds_max_nm > 0.0 ? ds_max_nm : 0.25 * g->h;
  try {
    // host side: argument checks and the segment index (vertex pairs), nothing else
    std::vector<int> first(n_lines + 1, 0), flag(n_lines), seg_line;
    std::vector<int2> seg;
    double sub = 0.0;
    for (int l = 0; l < n_lines; ++l) {
      if (counts[l] < 2 || (closed[l] != 0 && closed[l] != 1) || (closed[l] && counts[l] < 3))
        return fail(g, OKMC_EINVAL, "a line needs 2 vertices (3 when closed) and closed in {0, 1}");
      if ((long long)first[l] + counts[l] > (1ll << 28)) return fail(g, OKMC_EINVAL, "too many vertices");
      first[l + 1] = first[l] + counts[l];
      flag[l] = closed[l];
      for (int a = 0; a < 3; ++a)
        if (!std::isfinite(burgers[3 * l + a])) return fail(g, OKMC_EINVAL, "non-finite Burgers vector");
    }
    const int np = first[n_lines];
    for (long long k = 0; k < 3ll * np; ++k)
      if (!std::isfinite(points[k]) || std::fabs(points[k]) > 1e9) return fail(g, OKMC_EINVAL, "non-finite vertex");
    for (int l = 0; l < n_lines; ++l) {
      const int a0 = first[l], a1 = first[l + 1];
      const int ns = closed[l] ? counts[l] : counts[l] - 1;
      for (int k = 0; k < ns; ++k) {
        const int a = a0 + k, b = (a + 1 < a1) ? a + 1 : a0;
        const double dx = points[3 * b] - points[3 * a], dy = points[3 * b + 1] - points[3 * a + 1],
                     dz = points[3 * b + 2] - points[3 * a + 2];
        const double L = std::sqrt(dx * dx + dy * dy + dz * dz);
        if (!(L > 0.0)) return fail(g, OKMC_EINVAL, "zero-length segment");
        sub += std::ceil(L / ds) + 1.0;
        seg.push_back(make_int2(a, b));
        seg_line.push_back(l);
      }
    }
    if (sub > 1e9 || seg.size() > 0x7fffffffu) return fail(g, OKMC_EINVAL, "too many sub-segments");
    cudaStreamSynchronize(g->st);
    drop_graphs(g);
    g->gen += 1;
    dfree(g, g->d_bg);
    g->d_bg = nullptr;
    if (n_lines == 0) {
      OKMC_TRY(voxelise_all(g));
      return check_device_error(g);
    }
    const size_t N = g->N;
    const size_t nspec = 9 * (size_t)g->n[2] * g->P * 2 * tsize(g);
    const int tw = fp64(g) ? fdm_pencil_tile<double>(g->n[1], g->n[2], kSmemLimit)
                           : fdm_pencil_tile<float>(g->n[1], g->n[2], kSmemLimit);
    if (!tw) return fail(g, OKMC_EINVAL, "no pencil tile fits shared memory");
    double *d_pts = nullptr, *d_b = nullptr, *d_area = nullptr;
    int2* d_seg = nullptr;
    int *d_segl = nullptr, *d_first = nullptr, *d_closed = nullptr;
    unsigned long long* d_aq = nullptr;
    void* d_spec = nullptr;
    auto release = [&] {
      void* t[] = {d_pts, d_b, d_area, d_seg, d_segl, d_first, d_closed, d_aq, d_spec};
      for (void* p : t) dfree(g, p);
    };
    int rc = OKMC_OK;
    auto bail = [&](int code) {  // the error is reported once: the device flag is cleared
      release();
      dfree(g, g->d_bg);
      g->d_bg = nullptr;
      cudaMemsetAsync(g->d_err, 0, sizeof(int), g->st);
      voxelise_all(g);
      return code;
    };
    if ((rc = dalloc(g, (void**)&d_pts, 3 * (size_t)np * sizeof(double))) ||
        (rc = dalloc(g, (void**)&d_b, 3 * (size_t)n_lines * sizeof(double))) ||
        (rc = dalloc(g, (void**)&d_area, 3 * (size_t)n_lines * sizeof(double))) ||
        (rc = dalloc(g, (void**)&d_seg, seg.size() * sizeof(int2))) ||
        (rc = dalloc(g, (void**)&d_segl, seg.size() * sizeof(int))) ||
        (rc = dalloc(g, (void**)&d_first, first.size() * sizeof(int))) ||
        (rc = dalloc(g, (void**)&d_closed, flag.size() * sizeof(int))) ||
        (rc = dalloc(g, (void**)&d_aq, 9 * N * sizeof(unsigned long long))) || (rc = dalloc(g, &d_spec, nspec)) ||
        (rc = dalloc(g, &g->d_bg, 6 * N * qsize(g))))
      return bail(rc);
    cudaError_t e = cudaMemcpyAsync(d_pts, points, 3 * (size_t)np * sizeof(double), cudaMemcpyHostToDevice, g->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_b, burgers, 3 * (size_t)n_lines * sizeof(double), cudaMemcpyHostToDevice, g->st);
    if (e == cudaSuccess && !seg.empty())
      e = cudaMemcpyAsync(d_seg, seg.data(), seg.size() * sizeof(int2), cudaMemcpyHostToDevice, g->st);
    if (e == cudaSuccess && !seg.empty())
      e = cudaMemcpyAsync(d_segl, seg_line.data(), seg_line.size() * sizeof(int), cudaMemcpyHostToDevice, g->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_first, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice, g->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_closed, flag.data(), flag.size() * sizeof(int), cudaMemcpyHostToDevice, g->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_err, 0, sizeof(int), g->st);
    if (e != cudaSuccess) {
      cuda_fail(g, e, "dislocation upload");
      return bail(OKMC_ECUDA);
    }
    rc = run(g, "dislocation_eigenstrain", [&] {
      if (fp64(g))
        return launch_dislocation_eigenstrain<double, int64_t>(d_pts, d_seg, d_segl, (int)seg.size(), d_first, d_closed, d_b,
                                                               d_area, n_lines, ds, g->cfg, g->h, tw, d_aq,
                                                               (C2<double>*)d_spec, (int64_t*)g->d_bg, quantum(g), qlimit(g),
                                                               g->d_err, g->st);
      return launch_dislocation_eigenstrain<float, int32_t>(d_pts, d_seg, d_segl, (int)seg.size(), d_first, d_closed, d_b,
                                                            d_area, n_lines, ds, g->cfg, g->h, tw, d_aq,
                                                            (C2<float>*)d_spec, (int32_t*)g->d_bg, quantum(g), qlimit(g),
                                                            g->d_err, g->st);
    });
    if (rc) return bail(rc);
    if ((rc = check_device_error(g))) return bail(rc);
    release();
    OKMC_TRY(voxelise_all(g));
    return check_device_error(g);
  } catch (const std::bad_alloc&) {
    return fail(g, OKMC_ENOMEM, "host allocation failed");
  }
}

int okmc_point_dipole_energies(okmc_grid* g, const int32_t* pos, const double* P, int32_t m, double* E, int on_device) {
  if (!g || m < 0 || (m > 0 && (!pos || !P || !E))) return OKMC_EINVAL;
  if (m == 0) return OKMC_OK;
  std::lock_guard<std::recursive_mutex> lk(g_capture_mu);  // may allocate
  if (!on_device) {
    for (int k = 0; k < m; ++k) {
      const int32_t* p = pos + 3 * k;
      for (int a = 0; a < 3; ++a)
        if (p[a] < 0 || p[a] >= 2 * g->n[a]) return fail(g, OKMC_EINVAL, "probe site outside the box");
      if (((p[0] ^ p[1]) & 1) || ((p[0] ^ p[2]) & 1)) return fail(g, OKMC_EINVAL, "probe site off the bcc lattice");
      for (int a = 0; a < 6; ++a)
        if (!std::isfinite(P[6 * k + a])) return fail(g, OKMC_EINVAL, "non-finite dipole tensor");
    }
  }
  OKMC_TRY(solve(g));
  const int32_t* dpos = pos;
  const double* dP = P;
  double* dE = E;
  void *tpos = nullptr, *tP = nullptr, *tE = nullptr;
  auto release = [&] {
    if (tpos || tP || tE) cudaStreamSynchronize(g->st);
    dfree(g, tpos);
    dfree(g, tP);
    dfree(g, tE);
  };
  if (!on_device) {
    int rc = OKMC_OK;
    if ((rc = dalloc(g, &tpos, 3 * (size_t)m * sizeof(int32_t))) || (rc = dalloc(g, &tP, 6 * (size_t)m * sizeof(double))) ||
        (rc = dalloc(g, &tE, (size_t)m * sizeof(double)))) {
      release();
      return rc;
    }
    cudaError_t e = cudaMemcpyAsync(tpos, pos, 3 * (size_t)m * sizeof(int32_t), cudaMemcpyHostToDevice, g->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tP, P, 6 * (size_t)m * sizeof(double), cudaMemcpyHostToDevice, g->st);
    if (e != cudaSuccess) {
      release();
      return cuda_fail(g, e, "probe upload");
    }
    dpos = (const int32_t*)tpos;
    dP = (const double*)tP;
    dE = (double*)tE;
  }
  int rc = run(g, "point_dipole", [&] {
    if (fp64(g))
      return launch_point_dipole<double>((const double*)g->sig, dims(g), dpos, dP, m, g->cfg.C11, g->cfg.C12, g->cfg.C44, dE,
                                         g->d_err, g->st);
    return launch_point_dipole<float>((const float*)g->sig, dims(g), dpos, dP, m, g->cfg.C11, g->cfg.C12, g->cfg.C44, dE,
                                      g->d_err, g->st);
  });
  if (rc == OKMC_OK && !on_device) rc = copy_out(g, E, dE, (size_t)m * sizeof(double), 0);
  release();
  if (rc) return rc;
  int code = 0;
  cudaError_t e = cudaMemcpyAsync(&code, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
  if (e != cudaSuccess) return cuda_fail(g, e, "device error check");
  if (code == 8) {  // a device-side probe was rejected: report it and clear the flag
    if (cudaMemsetAsync(g->d_err, 0, sizeof(int), g->st) != cudaSuccess) return fail(g, OKMC_ECUDA, "error reset");
    return fail(g, OKMC_EINVAL, "probe site off the bcc lattice or outside the box");
  }
  return check_device_error(g);
}

}  // extern "C"

namespace {
template <class T, class Q>
int shift_energies(okmc_grid* g, int i, const double* dX, int m, double* dE) {
  const size_t N = g->N;
  const size_t sp = (size_t)g->n[2] * g->P * 2 * sizeof(T);  // one component of half spectrum
  void *spec_e = nullptr, *spec_w = nullptr, *fw = nullptr;
  auto release = [&] {
    cudaStreamSynchronize(g->st);
    dfree(g, spec_e);
    dfree(g, spec_w);
    dfree(g, fw);
  };
  int rc = OKMC_OK;
  if ((rc = dalloc(g, &spec_e, 6 * sp)) || (rc = dalloc(g, &spec_w, 2 * sp)) || (rc = dalloc(g, &fw, 2 * N * sizeof(Q)))) {
    release();
    return rc;
  }
  PassCfg c = g->cfg;
  c.forward_only = 1;
  c.dirty = nullptr;
  // the grid's eigenstrain, transformed
  c.q = quantum(g);
  c.ncomp = 6;
  rc = run(g, "shift_eps_fwd", [&] { return launch_plane_fwd<T, Q>((const Q*)g->eps, (C2<T>*)spec_e, c, g->st); });
  if (!rc) rc = run(g, "shift_eps_pencil", [&] { return launch_pencil<T>((C2<T>*)spec_e, c, g->st); });
  // the count fields of defect i's two stencils with their base voxel at the origin
  if (!rc && cudaMemsetAsync(fw, 0, 2 * N * sizeof(Q), g->st) != cudaSuccess) rc = fail(g, OKMC_ECUDA, "memset");
  WBatch b{};
  b.nb = 1;
  b.idx[0] = i;
  if (!rc) rc = run(g, "shift_fields", [&] { return launch_wfields<Q>((Q*)fw, dims(g), g->d_ptr, g->d_off, g->d_cnt, b, g->st); });
  c.q = 1.0;
  c.ncomp = 2;
  if (!rc) rc = run(g, "shift_w_fwd", [&] { return launch_plane_fwd<T, Q>((const Q*)fw, (C2<T>*)spec_w, c, g->st); });
  if (!rc) rc = run(g, "shift_w_pencil", [&] { return launch_pencil<T>((C2<T>*)spec_w, c, g->st); });
  c.ncomp = 6;
  const int per = shift_positions_per_pass();
  for (int k0 = 0; k0 < m && !rc; k0 += per) {
    const int mk = std::min(per, m - k0);
    rc = run(g, "shift_energies", [&] {
      return launch_shift_energies<T>((const C2<T>*)spec_e, (const C2<T>*)spec_w, c, g->d_def, g->d_geo, g->d_alpha, i,
                                      dX + 3 * (size_t)k0, mk, g->h, g->d_partial, kSelfBlocks, dE + k0, g->st);
    });
  }
  release();
  return rc;
}
}  // namespace

extern "C" {

int okmc_shift_energies(okmc_grid* g, int32_t i, const double* X, int32_t m, double* E, int on_device) {
  if (!g || m < 0 || (m > 0 && (!X || !E))) return OKMC_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(g_capture_mu);  // allocates
  if (i < 0 || i >= g->nd) return fail(g, OKMC_EINVAL, "defect index out of range");
  if (m == 0) return OKMC_OK;
  if (!on_device)
    for (long long k = 0; k < 3ll * m; ++k)
      if (!std::isfinite(X[k]) || std::fabs(X[k]) > 1e9) return fail(g, OKMC_EINVAL, "non-finite position");
  const double* dX = X;
  double* dE = E;
  void *tX = nullptr, *tE = nullptr;
  auto release = [&] {
    if (tX || tE) cudaStreamSynchronize(g->st);
    dfree(g, tX);
    dfree(g, tE);
  };
  if (!on_device) {
    int rc = OKMC_OK;
    if ((rc = dalloc(g, &tX, 3 * (size_t)m * sizeof(double))) || (rc = dalloc(g, &tE, (size_t)m * sizeof(double)))) {
      release();
      return rc;
    }
    cudaError_t e = cudaMemcpyAsync(tX, X, 3 * (size_t)m * sizeof(double), cudaMemcpyHostToDevice, g->st);
    if (e != cudaSuccess) {
      release();
      return cuda_fail(g, e, "position upload");
    }
    dX = (const double*)tX;
    dE = (double*)tE;
  }
  int rc = fp64(g) ? shift_energies<double, int64_t>(g, i, dX, m, dE) : shift_energies<float, int32_t>(g, i, dX, m, dE);
  if (!rc && !on_device) rc = copy_out(g, E, dE, (size_t)m * sizeof(double), 0);
  release();
  if (rc) return rc;
  return check_device_error(g);
}

int okmc_self_terms(okmc_grid* g, double* W, int out_on_device) {
  if (!g || !W) return OKMC_EINVAL;
  if (!g->nd) return OKMC_OK;
  return copy_out(g, W, g->d_W, g->nd * 18 * sizeof(double), out_on_device);
}

int okmc_get_stencil(okmc_grid* g, int32_t i, int32_t c, int32_t* offs, int32_t* counts, int32_t capacity, int32_t* k,
                     double* alpha) {
  if (!g || i < 0 || i >= g->nd || c < 0 || c > 1 || !k) return OKMC_EINVAL;
  int p[2];
  cudaError_t e = cudaMemcpyAsync(p, g->d_ptr + 2 * i + c, 2 * sizeof(int), cudaMemcpyDeviceToHost, g->st);
  double a = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&a, g->d_alpha + 2 * i + c, sizeof(double), cudaMemcpyDeviceToHost, g->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
  if (e != cudaSuccess) return cuda_fail(g, e, "stencil query");
  *k = p[1] - p[0];
  if (alpha) *alpha = a;
  if (capacity <= 0) return OKMC_OK;
  if (capacity < *k || !offs || !counts) return fail(g, OKMC_EINVAL, "capacity too small");
  std::vector<int> o(*k);
  std::vector<uint8_t> cn(*k);
  e = cudaMemcpyAsync(o.data(), g->d_off + p[0], *k * sizeof(int), cudaMemcpyDeviceToHost, g->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cn.data(), g->d_cnt + p[0], *k, cudaMemcpyDeviceToHost, g->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
  if (e != cudaSuccess) return cuda_fail(g, e, "stencil copy");
  for (int q = 0; q < *k; ++q) {
    unpack_off(o[q], offs[3 * q], offs[3 * q + 1], offs[3 * q + 2]);
    counts[q] = cn[q];
  }
  return OKMC_OK;
}

int okmc_get_stats(okmc_grid* g, okmc_step_stats* out) {
  if (!g || !out) return OKMC_EINVAL;
  DevState s;
  int derr = 0;
  cudaError_t e = cudaMemcpyAsync(&s, g->d_state, sizeof(s), cudaMemcpyDeviceToHost, g->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&derr, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
  if (e != cudaSuccess) return cuda_fail(g, e, "stats");
  if (derr) return check_device_error(g);
  out->events = s.events;
  out->steps = s.step;
  out->solves = g->solves;
  out->negative_barriers = s.negative_barriers;
  out->clock = s.clock;
  out->dt_last = s.dt_last;
  if (s.err) return fail(g, OKMC_ESTATE, "no mobile defect with a positive rate");
  return OKMC_OK;
}

int okmc_set_kinetic_state(okmc_grid* g, const okmc_step_stats* s) {
  if (!g || !s) return OKMC_EINVAL;
  if (s->events < 0 || s->steps < 0 || s->solves < 0 || s->negative_barriers < 0 || !std::isfinite(s->clock) ||
      !std::isfinite(s->dt_last))
    return fail(g, OKMC_EINVAL, "bad kinetic state");
  DevState st;
  cudaError_t e = cudaMemcpyAsync(&st, g->d_state, sizeof(st), cudaMemcpyDeviceToHost, g->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
  if (e != cudaSuccess) return cuda_fail(g, e, "state read");
  st.clock = s->clock;
  st.dt_last = s->dt_last;
  st.events = s->events;
  st.negative_barriers = s->negative_barriers;
  st.step = s->steps;
  e = cudaMemcpyAsync(g->d_state, &st, sizeof(st), cudaMemcpyHostToDevice, g->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
  if (e != cudaSuccess) return cuda_fail(g, e, "state write");
  g->solves = s->solves;
  return OKMC_OK;
}

int okmc_step(okmc_grid* g, const okmc_step_params* p, int64_t n_steps, okmc_step_stats* out) {
  if (!g || !p) return OKMC_EINVAL;
  if (!(p->T_K > 0.0) || !std::isfinite(p->T_K)) return fail(g, OKMC_EINVAL, "temperature must be > 0");
  if (p->mode != OKMC_RESIDENCE && p->mode != OKMC_FIXED_DT) return fail(g, OKMC_EINVAL, "unknown mode");
  if (n_steps < 0) return fail(g, OKMC_EINVAL, "negative step count");
  if (!g->nd || !g->any_mobile) return fail(g, OKMC_ESTATE, "no mobile defect");
  const double kT = kBoltzmann * p->T_K;
  // Steady state: replay a captured graph of the step (one launch per step).  With
  // kernel timing on, launch kernel by kernel so that each one can be timed.
  cudaGraphExec_t exec = nullptr;
  if (g->use_graphs && !g->profiling && n_steps > 0) {
    for (auto& s : g->graphs)
      if (s.mode == p->mode && s.T == p->T_K) exec = s.exec;
    if (!exec) {
      OKMC_TRY(capture_step(g, p->mode, p->T_K, &exec));
      g->graphs.push_back({p->mode, p->T_K, exec});
    }
  }
  for (int64_t s = 0; s < n_steps; ++s) {
    if (exec) {
      cudaError_t e = cudaGraphLaunch(exec, g->st);
      if (e != cudaSuccess) return cuda_fail(g, e, "graph launch");
      g->solves += 1;
      g->sigma_valid = false;
    } else {
      OKMC_TRY(step_body(g, p->mode, kT, false));
    }
    if (p->t_end > 0.0) {
      okmc_step_stats tmp;
      OKMC_TRY(okmc_get_stats(g, &tmp));
      if (tmp.clock >= p->t_end) break;
    }
  }
  if (out) OKMC_TRY(okmc_get_stats(g, out));
  return OKMC_OK;
}

int okmc_set_graphs(okmc_grid* g, int enable) {
  if (!g) return OKMC_EINVAL;
  g->use_graphs = enable != 0;
  return OKMC_OK;
}

// ---------------------------------------------------------------- batches
int okmc_batch_create(okmc_grid* const* grids, int32_t n, void* stream, okmc_batch** out) {
  if (!grids || n <= 0 || !out) return OKMC_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!grids[i]) return OKMC_EINVAL;
  okmc_batch* b = new (std::nothrow) okmc_batch();
  if (!b) return OKMC_ENOMEM;
  b->grids.assign(grids, grids + n);
  b->st = (cudaStream_t)stream;
  *out = b;
  return OKMC_OK;
}

int okmc_batch_destroy(okmc_batch* b) {
  if (!b) return OKMC_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto s : b->side) cudaStreamDestroy(s);
  for (auto e : b->ev) cudaEventDestroy(e);
  if (b->d_reps || b->d_items) {
    std::lock_guard<std::recursive_mutex> lk(g_capture_mu);
    cudaFree(b->d_reps);
    cudaFree(b->d_items);
  }
  release_slots(b);
  delete b;
  return OKMC_OK;
}

int okmc_batch_set_mode(okmc_batch* b, int32_t mode) {
  if (!b || (mode != OKMC_BATCH_AUTO && mode != OKMC_BATCH_KERNELS && mode != OKMC_BATCH_GRAPHS)) return OKMC_EINVAL;
  if (mode != b->mode) {
    b->mode = mode;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return OKMC_OK;
}

int okmc_batch_get_mode(const okmc_batch* b, int32_t* mode) {
  if (!b || !mode) return OKMC_EINVAL;
  *mode = b->used;
  return OKMC_OK;
}

const char* okmc_batch_last_error(const okmc_batch* b) { return b ? b->err.c_str() : "null batch"; }

static bool batch_kernels_ok(const okmc_batch* b) {
  for (const okmc_grid* g : b->grids)
    if (fp64(g) || !g->fast || !batch_edge_supported(g->n[0], g->n[1], g->n[2]) || !g->d_order ||
        (g->nd > 0 && g->nchunk == 0))
      return false;
  return true;
}

// The batched-kernel form: one record per replica and work lists uploaded once; the
// graph of a step holds, for each solve pass and edge class, one persistent launch over the
// planes (tiles) of every replica of that edge, then over every replica the energies and
// rates, the event and the field update (one persistent or one-block-per-replica launch
// each).
static int batch_build_kernels(okmc_batch* b) {
  const int n = (int)b->grids.size();
  std::vector<BatchRep> reps(n);
  for (int i = 0; i < n; ++i) {
    okmc_grid* g = b->grids[i];
    const okmc_step_params& p = b->params[i];
    BatchRep& r = reps[i];
    r.cfg = g->cfg;
    r.cfg.q = quantum(g);
    r.cfg.ncomp = 6;
    r.cfg.forward_only = 0;
    r.cfg.dirty = g->d_dirty;
    r.eps = (const int32_t*)g->eps;
    r.spec = (C2<float>*)g->spec;
    r.spec2 = (C2<float>*)g->spec2;
    r.sig = (float*)g->sig;
    r.def = g->d_def;
    r.geo = g->d_geo;
    r.ptr = g->d_ptr;
    r.off = g->d_off;
    r.cnt = g->d_cnt;
    r.alpha = g->d_alpha;
    r.W = g->d_W;
    r.order = g->d_order;
    r.E = g->d_E;
    r.Ec = g->d_Ec;
    const double kT = kBoltzmann * p.T_K;
    r.ra.rates = g->d_rates;
    r.ra.rsum = g->d_rsum;
    r.ra.negb = &g->d_state->negative_barriers;
    r.ra.nu0 = g->nu0;
    r.ra.kT = kT;
    r.ra.rkT = 1.0 / kT;
    if (g->d_dl) r.dl = DilatedLists{g->d_dl, g->d_dl + 2 * g->nd, g->d_doff, g->d_dcnt, g->d_dscnt};
    r.ca = ChunkArgs{g->d_cdef, g->d_c0, g->d_cpart, g->nchunk};
    r.pref = -kKappa * g->h * g->h * g->h;
    r.nu0 = g->nu0;
    r.kT = kT;
    r.moves = g->d_moves;
    r.state = g->d_state;
    r.err = g->d_err;
    r.rq = 1.0 / quantum(g);
    r.lim = qlimit(g);
    r.key0 = (uint32_t)g->desc.seed;
    r.key1 = (uint32_t)(g->desc.seed >> 32);
    r.n = dims(g);
    r.nd = g->nd;
    r.mode = p.mode;
  }
  // work lists: per edge class (ny, nz) its planes and its tiles, then every replica's defects
  struct Cls {
    int ny, nz;
    int plane0, nplane, tile0, ntile;
  };
  std::map<std::pair<int, int>, std::vector<int>> by_edge;
  for (int i = 0; i < n; ++i) by_edge[{b->grids[i]->n[1], b->grids[i]->n[2]}].push_back(i);
  std::vector<int2> items;
  std::vector<Cls> cls;
  for (const auto& kv : by_edge) {
    Cls c{kv.first.first, kv.first.second, (int)items.size(), 0, 0, 0};
    for (int i : kv.second)
      for (int k = 0; k < 6 * b->grids[i]->n[2]; ++k) items.push_back(make_int2(i, k));
    c.nplane = (int)items.size() - c.plane0;
    c.tile0 = (int)items.size();
    for (int i : kv.second)
      for (int k = 0; k < (int)(b->grids[i]->P / 8); ++k) items.push_back(make_int2(i, k));
    c.ntile = (int)items.size() - c.tile0;
    cls.push_back(c);
  }
  // energies: every replica's chunk slots, then its warps of three defects
  const int e0 = (int)items.size();
  for (int i = 0; i < n; ++i)
    for (int w = 0; w < b->grids[i]->nchunk; ++w) items.push_back(make_int2(i, w));
  const int ne = (int)items.size() - e0;
  const int f0 = (int)items.size();
  for (int i = 0; i < n; ++i)
    for (int q = 0; 3 * q < b->grids[i]->nd; ++q) items.push_back(make_int2(i, q));
  const int nf = (int)items.size() - f0;
  cudaFree(b->d_reps);
  cudaFree(b->d_items);
  b->d_reps = nullptr;
  b->d_items = nullptr;
  release_slots(b);
  b->slot0 = acquire_slots(n);
  if (b->slot0 < 0) {
    b->err = "batched kernels: more replicas in batches at once than the " + std::to_string(batch_cfg_slots()) +
             " configuration slots";
    return OKMC_ENOMEM;
  }
  b->nslots = n;
  std::vector<PassCfg> cfgs(n);
  for (int i = 0; i < n; ++i) cfgs[i] = reps[i].cfg;
  cudaError_t e = upload_batch_cfg(b->slot0, cfgs.data(), n, b->side[n]);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_reps, n * sizeof(BatchRep));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_items, items.size() * sizeof(int2));
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_reps, reps.data(), n * sizeof(BatchRep), cudaMemcpyHostToDevice, b->side[n]);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, b->side[n]);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->side[n]);
  if (e != cudaSuccess) {
    b->err = std::string("batch work lists: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? OKMC_ENOMEM : OKMC_ECUDA;
  }
  // grids (one CTA, or cluster, per item of the class's list) and kernel attributes
  // before the capture
  std::vector<std::array<int, 3>> grids(cls.size());
  for (size_t k = 0; k < cls.size(); ++k) {
    const Cls& c = cls[k];
    for (int pass = 0; pass < 3; ++pass) {
      grids[k][pass] = pass_batch_grid(pass, pass == 1 ? c.nz : c.ny, pass == 1 ? c.ntile : c.nplane);
      if (grids[k][pass] <= 0) {
        b->err = "batched kernels: no resident grid";
        return OKMC_ECUDA;
      }
    }
  }
  const int egrid = energies_batch_grid();  // resident blocks of 8 warps (one item per warp)
  while ((int)b->side.size() < n + 1 + (int)cls.size()) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return OKMC_ECUDA;
    b->side.push_back(st);
  }
  while ((int)b->ev.size() < 2 * n + 1 + (int)cls.size()) {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return OKMC_ECUDA;
    b->ev.push_back(ev);
  }
  cudaStream_t root = b->side[n];
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return OKMC_ECUDA;
  const int2* it = b->d_items;
  e = cudaSuccess;
  // each pass: the edge classes as parallel branches (a class's tail overlaps the
  // others' blocks), joined before the next pass
  for (int pass = 0; pass < 3 && e == cudaSuccess; ++pass) {
    e = cudaEventRecord(b->ev[2 * n], root);
    for (size_t k = 0; k < cls.size() && e == cudaSuccess; ++k) {
      const Cls& c = cls[k];
      cudaStream_t sk = b->side[n + 1 + k];
      e = cudaStreamWaitEvent(sk, b->ev[2 * n], 0);
      if (e == cudaSuccess)
        e = pass == 1 ? launch_pass_batch(1, c.nz, b->d_reps, it + c.tile0, c.ntile, grids[k][1], b->slot0, sk)
                      : launch_pass_batch(pass, c.ny, b->d_reps, it + c.plane0, c.nplane, grids[k][pass], b->slot0, sk);
      if (e == cudaSuccess) e = cudaEventRecord(b->ev[2 * n + 1 + k], sk);
    }
    for (size_t k = 0; k < cls.size() && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(root, b->ev[2 * n + 1 + k], 0);
  }
  if (e == cudaSuccess) e = launch_energy_chunks_batch(b->d_reps, it + e0, ne, std::max(1, std::min(egrid, (ne + 7) / 8)), root);
  if (e == cudaSuccess) e = launch_energy_finish_batch(b->d_reps, it + f0, nf, std::max(1, std::min(egrid, (nf + 7) / 8)), root);
  if (e == cudaSuccess) e = launch_event_batch(b->d_reps, n, root);
  if (e == cudaSuccess) e = launch_moves_batch(b->d_reps, n, root);
  cudaError_t e2 = cudaStreamEndCapture(root, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    b->err = std::string("batched kernels capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
    return OKMC_ECUDA;
  }
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return OKMC_ECUDA;
  b->used = OKMC_BATCH_KERNELS;
  return OKMC_OK;
}

// One graph holds every replica's step as an independent branch (fork/join on
// private streams); each launch advances all replicas by one step, and their
// kernels overlap on the GPU.
static int batch_build(okmc_batch* b) {
  std::lock_guard<std::recursive_mutex> lk(g_capture_mu);
  const int n = (int)b->grids.size();
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  const bool kern_ok = batch_kernels_ok(b);
  if (b->mode == OKMC_BATCH_KERNELS && !kern_ok) {
    b->err = "batched kernels need FP32-field replicas with nx = ny and edges in {64, 96, 128, 160, 192, 256}";
    return OKMC_EINVAL;
  }
  while ((int)b->side.size() < n + 1) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return OKMC_ECUDA;
    b->side.push_back(s);
  }
  while ((int)b->ev.size() < 2 * n + 1) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return OKMC_ECUDA;
    b->ev.push_back(e);
  }
  if (b->mode != OKMC_BATCH_GRAPHS && kern_ok) return batch_build_kernels(b);
  cudaStream_t root = b->side[n];
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return OKMC_ECUDA;
  int rc = OKMC_OK;
  if (cudaEventRecord(b->ev[2 * n], root) != cudaSuccess) rc = OKMC_ECUDA;
  for (int i = 0; i < n && rc == OKMC_OK; ++i) {
    okmc_grid* g = b->grids[i];
    const okmc_step_params& p = b->params[i];
    if (cudaStreamWaitEvent(b->side[i], b->ev[2 * n], 0) != cudaSuccess) { rc = OKMC_ECUDA; break; }
    cudaStream_t keep = g->st;
    const bool prof = g->profiling;
    g->st = b->side[i];
    g->profiling = false;
    rc = step_body(g, p.mode, kBoltzmann * p.T_K, true);
    g->st = keep;
    g->profiling = prof;
    if (rc != OKMC_OK) {
      b->err = "replica " + std::to_string(i) + ": " + g->err;
      break;
    }
    if (cudaEventRecord(b->ev[i], b->side[i]) != cudaSuccess || cudaStreamWaitEvent(root, b->ev[i], 0) != cudaSuccess)
      rc = OKMC_ECUDA;
  }
  cudaError_t e = cudaStreamEndCapture(root, &graph);
  if (rc != OKMC_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return OKMC_ECUDA;
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e == cudaSuccess) b->used = OKMC_BATCH_GRAPHS;
  return e == cudaSuccess ? OKMC_OK : OKMC_ECUDA;
}

int okmc_batch_step(okmc_batch* b, const okmc_step_params* params, int64_t n_steps, okmc_step_stats* stats) {
  if (!b || !params || n_steps < 0) return OKMC_EINVAL;
  const int n = (int)b->grids.size();
  bool same = (int)b->params.size() == n;
  for (int i = 0; i < n; ++i) {
    const okmc_step_params& p = params[i];
    okmc_grid* g = b->grids[i];
    if (!(p.T_K > 0.0) || (p.mode != OKMC_RESIDENCE && p.mode != OKMC_FIXED_DT) || p.t_end != 0.0) {
      b->err = "replica " + std::to_string(i) + ": bad step parameters (t_end must be 0 in a batch)";
      return OKMC_EINVAL;
    }
    if (!g->nd || !g->any_mobile) {
      b->err = "replica " + std::to_string(i) + ": no mobile defect";
      return OKMC_ESTATE;
    }
    if (same && (b->params[i].mode != p.mode || b->params[i].T_K != p.T_K)) same = false;
    if ((int)b->gens.size() != n || b->gens[i] != g->gen) same = false;
  }
  if (!same || !b->exec) {
    b->params.assign(params, params + n);
    b->gens.resize(n);
    for (int i = 0; i < n; ++i) b->gens[i] = b->grids[i]->gen;
    const int rc = batch_build(b);
    if (rc != OKMC_OK) {
      if (b->err.empty()) b->err = "batch graph capture failed";
      return rc;
    }
  }
  // the replicas' own streams must not have work in flight that the batch could race
  for (auto* g : b->grids) cudaStreamSynchronize(g->st);
  for (int64_t s = 0; s < n_steps; ++s) {
    cudaError_t e = cudaGraphLaunch(b->exec, b->st);
    if (e != cudaSuccess) {
      b->err = std::string("graph launch: ") + cudaGetErrorString(e);
      return OKMC_ECUDA;
    }
  }
  if (cudaStreamSynchronize(b->st) != cudaSuccess) return OKMC_ECUDA;
  for (int i = 0; i < n; ++i) {
    okmc_grid* g = b->grids[i];
    g->solves += n_steps;
    g->sigma_valid = false;
    if (stats) {
      const int rc = okmc_get_stats(g, &stats[i]);
      if (rc != OKMC_OK) return rc;
    }
  }
  return OKMC_OK;
}

size_t okmc_device_bytes(const okmc_grid* g) { return g ? g->bytes : 0; }

int okmc_set_profiling(okmc_grid* g, int enable) {
  if (!g) return OKMC_EINVAL;
  drain_profile(g);
  g->profiling = enable != 0;
  return OKMC_OK;
}

int okmc_kernel_times(okmc_grid* g, const char** names, double* ms, int64_t* count, int cap) {
  if (!g) return OKMC_EINVAL;
  drain_profile(g);
  g->prof_names.clear();
  for (auto& kv : g->prof) g->prof_names.push_back(kv.first);
  int k = 0;
  for (auto& kv : g->prof) {
    if (k < cap) {
      if (names) names[k] = g->prof_names[k].c_str();
      if (ms) ms[k] = kv.second.first;
      if (count) count[k] = kv.second.second;
    }
    ++k;
  }
  return k;
}

int okmc_reset_kernel_times(okmc_grid* g) {
  if (!g) return OKMC_EINVAL;
  drain_profile(g);
  g->prof.clear();
  return OKMC_OK;
}

int okmc_get_variants(const okmc_grid* g, int32_t current[3], int32_t available[3]) {
  if (!g || !current || !available) return OKMC_EINVAL;
  for (int p = 0; p < 3; ++p) {
    current[p] = g->variant[p];
    available[p] = g->avail[p];
  }
  return OKMC_OK;
}

int okmc_set_variant(okmc_grid* g, int32_t pass, int32_t variant) {
  if (!g) return OKMC_EINVAL;
  if (pass < 0 || pass > 2 || variant < 0 || variant > 30 || !((g->avail[pass] >> variant) & 1))
    return fail(g, OKMC_EINVAL, "no such launch variant for this grid");
  cudaStreamSynchronize(g->st);
  drop_graphs(g);
  g->variant[pass] = variant;
  g->sigma_valid = false;
  return OKMC_OK;
}

int okmc_launch_shape(const okmc_grid* g, int32_t out[3]) {
  if (!g || !out) return OKMC_EINVAL;
  out[0] = g->fast ? -1 : g->cfg.cs;  // -1: register-FFT plane passes
  out[1] = (int32_t)(g->P / (g->fast ? 8 : g->cfg.tw_w));
  out[2] = g->fast ? -1 : g->cfg.cs;
  return OKMC_OK;
}

}  // extern "C"
