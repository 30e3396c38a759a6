// Batched ensemble: many independent DGSEM runs (each its own mesh, degree N,
// gas constants and time step) advanced together.  Members of equal N form a
// group; per stage each group runs three persistent kernels (lifting, face
// flux, volume + update) that walk a tile table spanning all of the group's
// members, and the whole nsteps sequence is captured in one CUDA graph.  Tile
// shapes (elements per block) and grid sizes per group come from an autotuner
// that times the candidates on the members' own data and caches its choice in
// a small text file keyed by GPU name, N and operator precision.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "dg_stage.cuh"

namespace dg {

template <typename R>
struct MemberDev {
  double* U;
  double* G;
  double* clock;              // {t, dt} of this member
  const R* metrics;
  const double* metrics64;
  R* grad;
  R* fstar;
  const R* facegeo;
  const int* elem_face;
  const int* elem_nbr;
  const FaceInfo* faces;
  const double* mms;          // manufactured-source phases (or null)
  int E, F;
  Gas gas;
  double inv_w0;
};

// ---------------------------------------------------------------------------
// Persistent kernels: a block takes tiles t = blockIdx.x, blockIdx.x +
// gridDim.x, ...; tile = (member, block index inside the member).
template <int N, typename R, int EPB>
__global__ void __launch_bounds__(Shape<N, EPB>::THREADS)
k_lift_ens(const MemberDev<R>* __restrict__ mem, int nmem, const int2* __restrict__ tiles, int ntiles,
           const double* __restrict__ Dg) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 tl = tiles[t];
    const MemberDev<R>& m = mem[dg_idx(tl.x, nmem, kSiteEnsMember)];
    lift_body<N, R, EPB>(m.U, m.metrics, m.elem_nbr, m.elem_face, Dg, m.grad, m.E, m.gas, m.inv_w0, tl.y);
    __syncthreads();
  }
}

template <int N, typename R>
__global__ void __launch_bounds__(128)
k_face_ens(const MemberDev<R>* __restrict__ mem, int nmem, const int2* __restrict__ tiles, int ntiles) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 tl = tiles[t];
    const MemberDev<R>& m = mem[dg_idx(tl.x, nmem, kSiteEnsMember)];
    face_body<N, R>(m.U, m.grad, m.faces, m.facegeo, m.fstar, m.F, m.E, m.gas, (long)tl.y * 128 + threadIdx.x);
  }
}

template <int N, typename R, int EPB>
__global__ void __launch_bounds__(VShape<N, EPB>::THREADS)
k_volume_ens(const MemberDev<R>* __restrict__ mem, int nmem, const int2* __restrict__ tiles, int ntiles,
             const double* __restrict__ Dg, double c_stage, double A, double B) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 tl = tiles[t];
    const MemberDev<R>& m = mem[dg_idx(tl.x, nmem, kSiteEnsMember)];
    StageArgs a{m.U, m.U, m.G, nullptr, m.clock, c_stage, A, B, 1};
    volume_body<N, R, EPB>(a, m.metrics, m.metrics64, m.grad, m.fstar, m.elem_face, m.mms, Dg, m.E, m.gas,
                           m.inv_w0, tl.y);
    __syncthreads();
  }
}

__global__ void k_ens_clock_advance(double* const* clocks, int n) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n) clocks[b][0] += clocks[b][1];
}

__global__ void k_ens_set_clocks(double* const* clocks, const double* tdt, int n) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n) { clocks[b][0] = tdt[2 * b]; clocks[b][1] = tdt[2 * b + 1]; }
}

// ---------------------------------------------------------------------------
// Launch variants of one group: EPB choice 0 = default tile, 1 = doubled tile.
struct GroupPlan {
  int epb_choice = 0;   // 0: default tile, 1: doubled tile, 2: per-member launches of the single-run kernels
  int vol_grid = 0, lift_grid = 0, face_grid = 0;
  bool tuned = false, from_cache = false;
};

template <int N, typename R, int EPB>
static cudaError_t set_vol_attr() {
  return cudaFuncSetAttribute(k_volume_ens<N, R, EPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)volume_smem_bytes<N, R, EPB>());
}

template <int N, typename R>
struct Epb2 {   // the doubled tile, if it still fits a block (<= 1024 threads, <= 227 KB smem)
  static constexpr int base = default_epb((N + 1) * (N + 1) * (N + 1));
  static constexpr int P = (N + 1) * (N + 1) * (N + 1);
  static constexpr bool ok = 2 * base * P <= 1024 && volume_smem_bytes<N, R, 2 * base>() + 64 <= 227 * 1024;
  static constexpr int value = ok ? 2 * base : base;
};

struct Group {
  int N = 0;
  // members the tile-table kernels (LGL split form, conforming mesh, no FV
  // elements) do not cover: Gauss nodes, mortars or FV elements at creation;
  // they run as single-member units with their own stage kernels
  bool single_only = false;
  std::vector<int> members;            // indices into the ensemble
  void* d_mem = nullptr;               // MemberDev<R>[members]
  int2* d_elem_tiles[2] = {nullptr, nullptr};   // per EPB choice
  int n_elem_tiles[2] = {0, 0};
  int2* d_face_tiles = nullptr;
  int n_face_tiles = 0;
  const double* d_D = nullptr;
  GroupPlan plan;
};

template <int N, typename R>
static cudaError_t launch_group_stage(const Group& g, int k, const double* A, const double* B, const double* C,
                                      cudaStream_t s) {
  constexpr int e0 = Shape<N>::EPB, e1 = Epb2<N, R>::value;
  const MemberDev<R>* mem = (const MemberDev<R>*)g.d_mem;
  const int ch = g.plan.epb_choice;
  // lifting always uses the default tile (its tile table is choice 0)
  const int nmem = (int)g.members.size();
  k_lift_ens<N, R, e0><<<g.plan.lift_grid, Shape<N, e0>::THREADS, lift_smem_bytes<N, R, e0>(), s>>>(
      mem, nmem, g.d_elem_tiles[0], g.n_elem_tiles[0], g.d_D);
  k_face_ens<N, R><<<g.plan.face_grid, 128, 0, s>>>(mem, nmem, g.d_face_tiles, g.n_face_tiles);
  if (ch == 0)
    k_volume_ens<N, R, e0><<<g.plan.vol_grid, VShape<N, e0>::THREADS, volume_smem_bytes<N, R, e0>(), s>>>(
        mem, nmem, g.d_elem_tiles[0], g.n_elem_tiles[0], g.d_D, C[k], A[k], B[k]);
  else
    k_volume_ens<N, R, e1><<<g.plan.vol_grid, VShape<N, e1>::THREADS, volume_smem_bytes<N, R, e1>(), s>>>(
        mem, nmem, g.d_elem_tiles[1], g.n_elem_tiles[1], g.d_D, C[k], A[k], B[k]);
  return cudaGetLastError();
}

template <int N, typename R>
static cudaError_t setup_group() {
  cudaError_t e = cudaFuncSetAttribute(k_lift_ens<N, R, Shape<N>::EPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)lift_smem_bytes<N, R, Shape<N>::EPB>());
  if (e == cudaSuccess) e = set_vol_attr<N, R, Shape<N>::EPB>();
  if (e == cudaSuccess) e = set_vol_attr<N, R, Epb2<N, R>::value>();
  return e;
}

template <typename R>
static cudaError_t dispatch_stage(const Group& g, int k, const double* A, const double* B, const double* C,
                                  cudaStream_t s) {
  switch (g.N) {
    case 1: return launch_group_stage<1, R>(g, k, A, B, C, s);
    case 2: return launch_group_stage<2, R>(g, k, A, B, C, s);
    case 3: return launch_group_stage<3, R>(g, k, A, B, C, s);
    case 4: return launch_group_stage<4, R>(g, k, A, B, C, s);
    case 5: return launch_group_stage<5, R>(g, k, A, B, C, s);
    case 6: return launch_group_stage<6, R>(g, k, A, B, C, s);
    case 7: return launch_group_stage<7, R>(g, k, A, B, C, s);
    case 8: return launch_group_stage<8, R>(g, k, A, B, C, s);
    case 9: return launch_group_stage<9, R>(g, k, A, B, C, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
static cudaError_t dispatch_setup(int N) {
  switch (N) {
    case 1: return setup_group<1, R>();
    case 2: return setup_group<2, R>();
    case 3: return setup_group<3, R>();
    case 4: return setup_group<4, R>();
    case 5: return setup_group<5, R>();
    case 6: return setup_group<6, R>();
    case 7: return setup_group<7, R>();
    case 8: return setup_group<8, R>();
    case 9: return setup_group<9, R>();
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
static int epb_of_t(int N, int choice) {
  switch (N) {
    case 1: return choice ? Epb2<1, R>::value : Shape<1>::EPB;
    case 2: return choice ? Epb2<2, R>::value : Shape<2>::EPB;
    case 3: return choice ? Epb2<3, R>::value : Shape<3>::EPB;
    case 4: return choice ? Epb2<4, R>::value : Shape<4>::EPB;
    case 5: return choice ? Epb2<5, R>::value : Shape<5>::EPB;
    case 6: return choice ? Epb2<6, R>::value : Shape<6>::EPB;
    case 7: return choice ? Epb2<7, R>::value : Shape<7>::EPB;
    case 8: return choice ? Epb2<8, R>::value : Shape<8>::EPB;
    case 9: return choice ? Epb2<9, R>::value : Shape<9>::EPB;
    default: return 1;
  }
}

static int epb_of(int N, int choice, int precision) {
  return precision == DG_FP32OP ? epb_of_t<float>(N, choice) : epb_of_t<double>(N, choice);
}

// Host reader of this file's bounds-check error word (0 in normal builds).
DG_BOUNDS_READER(bounds_word_ensemble)
DG_BULK_READER(bulk_word_ensemble)

}  // namespace dg

using namespace dg;

// Side streams of the ensemble graph: how many independent work units run as
// parallel branches within a step.
constexpr int kEnsembleBranches = 8;

struct dg_ensemble {
  std::vector<Ctx*> members;
  int device = 0;
  int precision = DG_FP64;
  RkScheme rk = rk_scheme(DG_RK45);   // the members' common time scheme
  std::vector<Group> groups;
  std::string cache_path;
  std::string gpu_name;
  int sms = 0;
  // per-member device tables
  double** d_G = nullptr;
  double** d_clocks = nullptr;
  size_t* d_len = nullptr;
  double* d_tdt = nullptr;
  double* h_tdt = nullptr;
  double* clocks = nullptr;       // device [n][2]
  std::vector<double*> cur_U, cur_G;
  cudaGraphExec_t graph = nullptr;
  int graph_nsteps = 0;
  std::vector<int> graph_fv;      // each member's FV mode when the graph was captured
  std::vector<cudaStream_t> branch;   // side streams of the captured graph's parallel branches
  std::string err;
  std::string plan_json;
};

static dg_status ens_fail(dg_ensemble* e, dg_status st, const char* what, cudaError_t ce = cudaSuccess) {
  char buf[512];
  if (ce != cudaSuccess) std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(ce));
  else std::snprintf(buf, sizeof buf, "%s", what);
  if (e) e->err = buf;
  return st;
}

#define ENS_CUDA(call, e, what)                                                  \
  do {                                                                           \
    cudaError_t _c = (call);                                                     \
    if (_c != cudaSuccess) return ens_fail(e, DG_ECUDA, what, _c);               \
  } while (0)

template <typename R>
static void fill_member(MemberDev<R>& m, Ctx* c, double* U, double* G, double* clock) {
  m.U = U;
  m.G = G;
  m.clock = clock;
  m.metrics = (const R*)(sizeof(R) == 8 ? (const void*)c->d_metrics : (const void*)c->d_metrics_f);
  m.metrics64 = c->d_metrics;
  m.grad = (R*)c->d_grad;
  m.fstar = (R*)c->d_fstar;
  m.facegeo = (const R*)(sizeof(R) == 8 ? (const void*)c->d_facegeo : (const void*)c->d_facegeo_f);
  m.elem_face = c->d_elem_face;
  m.elem_nbr = c->d_elem_nbr;
  m.faces = c->d_faces;
  m.mms = c->d_mms;
  m.E = c->E;
  m.F = c->nfaces;
  m.gas = c->gas;
  m.inv_w0 = 1.0 / c->w[0];
}

// Upload the member tables of every group for the given state/register pointers.
static dg_status upload_members(dg_ensemble* e) {
  for (Group& g : e->groups) {
    if (g.single_only) continue;   // no member table
    if (e->precision == DG_FP32OP) {
      std::vector<MemberDev<float>> h(g.members.size());
      for (size_t a = 0; a < g.members.size(); ++a) {
        const int r = g.members[a];
        fill_member(h[a], e->members[r], e->cur_U[r], e->cur_G[r], e->clocks + 2 * r);
      }
      ENS_CUDA(cudaMemcpy(g.d_mem, h.data(), sizeof(h[0]) * h.size(), cudaMemcpyHostToDevice), e, "member table");
    } else {
      std::vector<MemberDev<double>> h(g.members.size());
      for (size_t a = 0; a < g.members.size(); ++a) {
        const int r = g.members[a];
        fill_member(h[a], e->members[r], e->cur_U[r], e->cur_G[r], e->clocks + 2 * r);
      }
      ENS_CUDA(cudaMemcpy(g.d_mem, h.data(), sizeof(h[0]) * h.size(), cudaMemcpyHostToDevice), e, "member table");
    }
  }
  std::vector<double*> hG(e->members.size()), hC(e->members.size());
  for (size_t r = 0; r < e->members.size(); ++r) { hG[r] = e->cur_G[r]; hC[r] = e->clocks + 2 * r; }
  ENS_CUDA(cudaMemcpy(e->d_G, hG.data(), sizeof(double*) * hG.size(), cudaMemcpyHostToDevice), e, "G table");
  ENS_CUDA(cudaMemcpy(e->d_clocks, hC.data(), sizeof(double*) * hC.size(), cudaMemcpyHostToDevice), e, "clock table");
  return DG_OK;
}

// Per-member candidate: the single-run kernels of each member in turn (best
// when every member fills the GPU by itself).
static cudaError_t one_member_stage(dg_ensemble* e, int r, int k, const double* A, const double* B, cudaStream_t s) {
  const Ctx& c = *e->members[r];
  double* U = e->cur_U[r];
  cudaError_t err;
  if ((err = launch_fv_switch(c, U, s)) != cudaSuccess) return err;   // automatic DG/FV switching, if set
  if ((err = launch_lift(c, U, s, false)) != cudaSuccess) return err;
  if ((err = launch_face(c, U, s, false)) != cudaSuccess) return err;
  StageArgs a{U, U, e->cur_G[r], nullptr, e->clocks + 2 * r, e->rk.C[k], A[k], B[k], 1};
  return launch_volume(c, a, s, false);
}

static cudaError_t member_stage(dg_ensemble* e, const Group& g, int k, const double* A, const double* B,
                                cudaStream_t s) {
  cudaError_t err = cudaSuccess;
  for (int r : g.members)
    if ((err = one_member_stage(e, r, k, A, B, s)) != cudaSuccess) return err;
  return err;
}

static cudaError_t enqueue_group(dg_ensemble* e, const Group& g, int k, const double* A, const double* B,
                                 cudaStream_t s) {
  if (g.plan.epb_choice == 2) return member_stage(e, g, k, A, B, s);
  return e->precision == DG_FP32OP ? dispatch_stage<float>(g, k, A, B, e->rk.C, s)
                                   : dispatch_stage<double>(g, k, A, B, e->rk.C, s);
}

static cudaError_t enqueue_stage(dg_ensemble* e, const Group& g, int k, cudaStream_t s) {
  return enqueue_group(e, g, k, e->rk.A, e->rk.B, s);
}

// ---------------------------------------------------------------------------
// Autotuner: for every group, time the volume kernel for each (tile, grid)
// candidate and the lifting / face kernels for each grid, on the members' own
// data, with B = 0 so the state is left untouched (the register is zeroed at
// the start of every step anyway).
static const double kZero14[14] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};

static float time_stage(dg_ensemble* e, const Group& g, cudaStream_t s, int reps, int which) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const double* Bz = kZero14;
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a, s);
    cudaError_t err = enqueue_group(e, g, 0, e->rk.A, Bz, s);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (err != cudaSuccess) ms = 1e30f;
    best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  (void)which;
  return best;
}

static std::string cache_key(const dg_ensemble* e, int N) {
  char k[256];
  std::snprintf(k, sizeof k, "%s|N=%d|%s", e->gpu_name.c_str(), N, e->precision == DG_FP32OP ? "fp32op" : "fp64");
  return k;
}

static std::map<std::string, GroupPlan> read_cache(const std::string& path) {
  std::map<std::string, GroupPlan> m;
  if (path.empty()) return m;
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return m;
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    char key[256];
    GroupPlan p;
    if (std::sscanf(line, "%255[^\t]\t%d\t%d\t%d\t%d", key, &p.epb_choice, &p.vol_grid, &p.lift_grid,
                    &p.face_grid) == 5) {
      // a line that no tuning run writes (edited or damaged file) is ignored,
      // so that group is tuned again
      const bool per_member = p.epb_choice == 2;
      const bool tiles = (p.epb_choice == 0 || p.epb_choice == 1) && p.vol_grid > 0 && p.lift_grid > 0 &&
                         p.face_grid > 0;
      if (!per_member && !tiles) continue;
      p.tuned = true;
      p.from_cache = true;
      m[key] = p;
    }
  }
  std::fclose(f);
  return m;
}

static void write_cache(const std::string& path, const std::map<std::string, GroupPlan>& m) {
  if (path.empty()) return;
  std::string tmp = path + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  for (const auto& kv : m)
    std::fprintf(f, "%s\t%d\t%d\t%d\t%d\n", kv.first.c_str(), kv.second.epb_choice, kv.second.vol_grid,
                 kv.second.lift_grid, kv.second.face_grid);
  std::fclose(f);
  std::rename(tmp.c_str(), path.c_str());
}

static dg_status autotune(dg_ensemble* e, cudaStream_t s) {
  std::map<std::string, GroupPlan> cache = read_cache(e->cache_path);
  bool dirty = false;
  const int sms = e->sms;
  for (Group& g : e->groups) {
    if (g.single_only) continue;   // nothing to tune: per-member launches
    const std::string key = cache_key(e, g.N);
    auto it = cache.find(key);
    if (it != cache.end()) {
      // the key holds no member sizes: the cached grids may exceed this
      // group's tile counts (the persistent kernels would only idle there)
      g.plan = it->second;
      if (g.plan.epb_choice != 2) {
        g.plan.vol_grid = std::min(g.plan.vol_grid, g.n_elem_tiles[g.plan.epb_choice]);
        g.plan.lift_grid = std::min(g.plan.lift_grid, g.n_elem_tiles[0]);
        g.plan.face_grid = std::min(g.plan.face_grid, g.n_face_tiles);
      }
      continue;
    }
    GroupPlan best;
    float best_ms = 1e30f;
    const int grids[4] = {sms, 2 * sms, 4 * sms, 0};
    for (int ch = 0; ch < 2; ++ch) {
      if (ch == 1 && epb_of(g.N, 1, e->precision) == epb_of(g.N, 0, e->precision)) continue;
      for (int gi = 0; gi < 4; ++gi) {
        GroupPlan p;
        p.epb_choice = ch;
        p.vol_grid = grids[gi] ? std::min(grids[gi], g.n_elem_tiles[ch]) : g.n_elem_tiles[ch];
        p.lift_grid = grids[gi] ? std::min(grids[gi], g.n_elem_tiles[0]) : g.n_elem_tiles[0];
        p.face_grid = grids[gi] ? std::min(grids[gi], g.n_face_tiles) : g.n_face_tiles;
        Group trial = g;
        trial.plan = p;
        const float ms = time_stage(e, trial, s, 3, 0);
        if (ms < best_ms) { best_ms = ms; best = p; }
      }
    }
    {
      GroupPlan p;
      p.epb_choice = 2;
      Group trial = g;
      trial.plan = p;
      const float ms = time_stage(e, trial, s, 3, 0);
      if (ms < best_ms) { best_ms = ms; best = p; }
    }
    best.tuned = true;
    g.plan = best;
    cache[key] = best;
    dirty = true;
  }
  if (dirty) write_cache(e->cache_path, cache);
  // plan description
  std::string js = "{\"gpu\": \"" + e->gpu_name + "\", \"groups\": [";
  for (size_t a = 0; a < e->groups.size(); ++a) {
    const Group& g = e->groups[a];
    char buf[400];
    std::snprintf(buf, sizeof buf,
                  "%s{\"N\": %d, \"members\": %zu, \"mode\": \"%s\", \"elements_per_block\": %d, \"volume_grid\": %d, "
                  "\"lift_grid\": %d, \"face_grid\": %d, \"element_tiles\": %d, \"face_tiles\": %d, \"cached\": %s}",
                  a ? ", " : "", g.N, g.members.size(),
                  g.single_only ? "per-member launches (Gauss nodes, mortars or FV elements)"
                                : (g.plan.epb_choice == 2 ? "per-member launches" : "tile table"),
                  g.plan.epb_choice == 2 ? 0 : epb_of(g.N, g.plan.epb_choice, e->precision), g.plan.vol_grid,
                  g.plan.lift_grid, g.plan.face_grid, g.n_elem_tiles[g.plan.epb_choice == 1 ? 1 : 0], g.n_face_tiles,
                  g.plan.from_cache ? "true" : "false");
    js += buf;
  }
  js += "]}";
  e->plan_json = js;
  return DG_OK;
}

// `e` holds the ensemble under construction, so that the caller can free it
// if a host allocation throws half-way.
static dg_status ensemble_create_impl(dg_ctx* const* members, int32_t n, const char* tune_cache_path,
                                      dg_ensemble** out, dg_ensemble*& e) {
  if (out) *out = nullptr;
  if (!members || n < 1 || !out) return DG_EINVAL;
  e = new dg_ensemble();
  auto bail = [&](dg_status st) {   // frees the device buffers the groups hold so far
    dg_ensemble_destroy(e);
    e = nullptr;
    return st;
  };
  auto drop = [&](dg_status st) {   // before any device allocation
    delete e;
    e = nullptr;
    return st;
  };
  Ctx* c0 = reinterpret_cast<Ctx*>(members[0]);
  if (!c0) return drop(DG_EINVAL);
  e->device = c0->device;
  e->precision = c0->prm.precision;
  e->rk = rk_scheme(c0->prm.rk_scheme);
  e->cache_path = tune_cache_path ? tune_cache_path : "";
  std::set<const Ctx*> seen;
  for (int r = 0; r < n; ++r) {
    Ctx* c = reinterpret_cast<Ctx*>(members[r]);
    // a context twice would have two members share its work buffers
    if (!c || c->device != e->device || c->prm.precision != e->precision || !seen.insert(c).second)
      return drop(DG_EINVAL);
    if (c->prm.rk_scheme != c0->prm.rk_scheme)   // one time scheme for all members
      return drop(DG_EUNSUPPORTED);
    e->members.push_back(c);
  }
  if (cudaSetDevice(e->device) != cudaSuccess) return drop(DG_ECUDA);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, e->device) != cudaSuccess) return drop(DG_ECUDA);
  e->gpu_name = prop.name;
  e->sms = prop.multiProcessorCount;
  // the members of the tile-table kernels by N; the others by N as single-member units
  std::map<int, std::vector<int>> byN, singles;
  for (int r = 0; r < n; ++r) {
    const Ctx* c = e->members[r];
    if (c->prm.nodes == DG_NODES_LGL && c->M == 0 && !c->fv_on) byN[c->N].push_back(r);
    else singles[c->N].push_back(r);
  }
  for (auto& kv : singles) {
    e->groups.emplace_back();
    Group& g = e->groups.back();
    g.N = kv.first;
    g.members = kv.second;
    g.single_only = true;
    g.plan.epb_choice = 2;
    g.plan.tuned = true;
  }
  for (auto& kv : byN) {
    e->groups.emplace_back();   // owned by e from here on, so bail() frees what it holds
    Group& g = e->groups.back();
    g.N = kv.first;
    g.members = kv.second;
    g.d_D = e->members[g.members[0]]->d_D;
    const size_t msz = e->precision == DG_FP32OP ? sizeof(MemberDev<float>) : sizeof(MemberDev<double>);
    if (cudaMalloc(&g.d_mem, msz * g.members.size()) != cudaSuccess) return bail(DG_ENOMEM);
    for (int ch = 0; ch < 2; ++ch) {
      const int epb = epb_of(g.N, ch, e->precision);
      std::vector<int2> t;
      for (size_t a = 0; a < g.members.size(); ++a) {
        const int E = e->members[g.members[a]]->E;
        for (int b = 0; b < (E + epb - 1) / epb; ++b) t.push_back(make_int2((int)a, b));
      }
      g.n_elem_tiles[ch] = (int)t.size();
      if (cudaMalloc(&g.d_elem_tiles[ch], sizeof(int2) * t.size()) != cudaSuccess) return bail(DG_ENOMEM);
      if (cudaMemcpy(g.d_elem_tiles[ch], t.data(), sizeof(int2) * t.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(DG_ECUDA);
    }
    std::vector<int2> ft;
    const int NN = (g.N + 1) * (g.N + 1);
    for (size_t a = 0; a < g.members.size(); ++a) {
      const long tot = (long)e->members[g.members[a]]->nfaces * NN;
      for (int b = 0; b < (int)((tot + 127) / 128); ++b) ft.push_back(make_int2((int)a, b));
    }
    g.n_face_tiles = (int)ft.size();
    if (cudaMalloc(&g.d_face_tiles, sizeof(int2) * ft.size()) != cudaSuccess) return bail(DG_ENOMEM);
    if (cudaMemcpy(g.d_face_tiles, ft.data(), sizeof(int2) * ft.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(DG_ECUDA);
    cudaError_t ce = e->precision == DG_FP32OP ? dispatch_setup<float>(g.N) : dispatch_setup<double>(g.N);
    if (ce != cudaSuccess) return bail(DG_ECUDA);
  }
  if (cudaMalloc(&e->d_G, sizeof(double*) * n) != cudaSuccess ||
      cudaMalloc(&e->d_clocks, sizeof(double*) * n) != cudaSuccess ||
      cudaMalloc(&e->d_len, sizeof(size_t) * n) != cudaSuccess ||
      cudaMalloc(&e->d_tdt, sizeof(double) * 2 * n) != cudaSuccess ||
      cudaMalloc(&e->clocks, sizeof(double) * 2 * n) != cudaSuccess ||
      cudaMallocHost(&e->h_tdt, sizeof(double) * 2 * n) != cudaSuccess)
    return bail(DG_ENOMEM);
  std::vector<size_t> len(n);
  for (int r = 0; r < n; ++r) len[r] = (size_t)e->members[r]->E * 5 * e->members[r]->P;
  if (cudaMemcpy(e->d_len, len.data(), sizeof(size_t) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(DG_ECUDA);
  e->cur_U.assign(n, nullptr);
  e->cur_G.assign(n, nullptr);
  *out = e;
  return DG_OK;
}

extern "C" {

// Host containers (tile tables, member lists) may throw when host memory runs
// out; no exception leaves the C ABI.
dg_status dg_ensemble_create(dg_ctx* const* members, int32_t n, const char* tune_cache_path, dg_ensemble** out) {
  dg_ensemble* e = nullptr;
  try {
    return ensemble_create_impl(members, n, tune_cache_path, out, e);
  } catch (const std::bad_alloc&) {
    if (e) dg_ensemble_destroy(e);   // the half-built ensemble and its device buffers
    if (out) *out = nullptr;
    return DG_ENOMEM;
  }
}

dg_status dg_ensemble_destroy(dg_ensemble* e) {
  if (!e) return DG_EINVAL;
  cudaSetDevice(e->device);
  cudaDeviceSynchronize();
  if (e->graph) cudaGraphExecDestroy(e->graph);
  for (Group& g : e->groups) {
    if (g.d_mem) cudaFree(g.d_mem);
    for (int ch = 0; ch < 2; ++ch) if (g.d_elem_tiles[ch]) cudaFree(g.d_elem_tiles[ch]);
    if (g.d_face_tiles) cudaFree(g.d_face_tiles);
  }
  void* bufs[] = {e->d_G, e->d_clocks, e->d_len, e->d_tdt, e->clocks};
  for (void* p : bufs) if (p) cudaFree(p);
  for (cudaStream_t bs : e->branch) cudaStreamDestroy(bs);
  if (e->h_tdt) cudaFreeHost(e->h_tdt);
  delete e;
  return DG_OK;
}

dg_status dg_ensemble_step(dg_ensemble* e, double* const* dU, double* const* dG, const double* t, const double* dt,
                           int32_t nsteps, dg_stream stream) {
  if (!e || !dU || !dG || !t || !dt || nsteps < 0) return ens_fail(e, DG_EINVAL, "dg_ensemble_step: bad argument");
  if (nsteps == 0) return DG_OK;
  const int n = (int)e->members.size();
  for (const Group& g : e->groups)
    for (int r : g.members)
      if (!g.single_only && e->members[r]->fv_on)
        return ens_fail(e, DG_EUNSUPPORTED,
                        "dg_ensemble_step: a member got FV sub-cell elements after the ensemble was created");
  cudaStream_t s = (cudaStream_t)stream;
  ENS_CUDA(cudaSetDevice(e->device), e, "cudaSetDevice");
  bool changed = false;
  std::set<const double*> distinct;
  for (int r = 0; r < n; ++r) {
    if (!dU[r] || !dG[r] || !distinct.insert(dU[r]).second || !distinct.insert(dG[r]).second)
      return ens_fail(e, DG_EINVAL, "dg_ensemble_step: null or repeated state pointers");
    if (dU[r] != e->cur_U[r] || dG[r] != e->cur_G[r]) changed = true;
  }
  if (changed) {
    for (int r = 0; r < n; ++r) { e->cur_U[r] = dU[r]; e->cur_G[r] = dG[r]; }
    ENS_CUDA(cudaStreamSynchronize(s), e, "sync before table upload");
    dg_status st = upload_members(e);
    if (st != DG_OK) return st;
    if (e->graph) { cudaGraphExecDestroy(e->graph); e->graph = nullptr; }
  }
  // clocks: staged through a pinned buffer, copied and consumed in stream order
  ENS_CUDA(cudaStreamSynchronize(s), e, "sync before clock staging");
  for (int r = 0; r < n; ++r) { e->h_tdt[2 * r] = t[r]; e->h_tdt[2 * r + 1] = dt[r]; }
  ENS_CUDA(cudaMemcpyAsync(e->d_tdt, e->h_tdt, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, s), e, "clock copy");
  k_ens_set_clocks<<<(n + 127) / 128, 128, 0, s>>>(e->d_clocks, e->d_tdt, n);
  ENS_CUDA(cudaGetLastError(), e, "clock kernel");
  bool need_tune = e->plan_json.empty();
  for (const Group& g : e->groups) need_tune |= !g.plan.tuned;
  // a member's FV mode changes its own launch sequence: capture again
  std::vector<int> fv_now(n);
  for (int r = 0; r < n; ++r) fv_now[r] = (e->members[r]->fv_on ? 1 : 0) + (e->members[r]->fv_switch ? 2 : 0);
  if (e->graph && fv_now != e->graph_fv) { cudaGraphExecDestroy(e->graph); e->graph = nullptr; }
  if (need_tune) {
    ENS_CUDA(cudaStreamSynchronize(s), e, "sync before tuning");
    dg_status st = autotune(e, s);
    if (st != DG_OK) return st;
    ENS_CUDA(cudaStreamSynchronize(s), e, "sync after tuning");
  }
  if (!e->graph || e->graph_nsteps != nsteps) {
    if (e->graph) { cudaGraphExecDestroy(e->graph); e->graph = nullptr; }
    cudaStream_t cs;
    ENS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), e, "capture stream");
    cudaGraph_t gr = nullptr;
    // Independent work units: a tile-table group (all its members in one set
    // of launches) or one member of a per-member group.  Within a step the
    // units are parallel branches of the graph, dealt to the side streams by
    // size (largest first, to the least loaded), so that one unit's kernel
    // tails and launch gaps are filled by another's blocks.
    struct Unit { int g, r; double dof; };
    std::vector<Unit> units;
    for (size_t gi = 0; gi < e->groups.size(); ++gi) {
      const Group& g = e->groups[gi];
      if (g.plan.epb_choice == 2) {
        for (int r : g.members) units.push_back({(int)gi, r, (double)e->members[r]->E * e->members[r]->P});
      } else {
        double dof = 0;
        for (int r : g.members) dof += (double)e->members[r]->E * e->members[r]->P;
        units.push_back({(int)gi, -1, dof});
      }
    }
    std::sort(units.begin(), units.end(), [](const Unit& a, const Unit& b) { return a.dof > b.dof; });
    const int nb = std::max(1, std::min<int>(kEnsembleBranches, (int)units.size()));
    std::vector<std::vector<Unit>> lanes(nb);
    std::vector<double> load(nb, 0.0);
    for (const Unit& u : units) {
      const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      lanes[b].push_back(u);
      load[b] += u.dof;
    }
    cudaError_t err = cudaSuccess;
    while ((int)e->branch.size() < nb && err == cudaSuccess) {
      cudaStream_t bs;
      err = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
      if (err == cudaSuccess) e->branch.push_back(bs);
    }
    std::vector<cudaEvent_t> evs;
    auto event = [&](cudaEvent_t* ev) {
      cudaError_t ce = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
      if (ce == cudaSuccess) evs.push_back(*ev);
      return ce;
    };
    if (err == cudaSuccess) err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    for (int st = 0; st < nsteps && err == cudaSuccess; ++st) {
      cudaEvent_t fork;
      if ((err = event(&fork)) != cudaSuccess || (err = cudaEventRecord(fork, cs)) != cudaSuccess) break;
      for (int b = 0; b < nb && err == cudaSuccess; ++b) {
        cudaStream_t bs = e->branch[b];
        err = cudaStreamWaitEvent(bs, fork, 0);
        for (const Unit& u : lanes[b]) {
          const Group& g = e->groups[u.g];
          for (int r : g.members) {
            if (err != cudaSuccess || (u.r >= 0 && r != u.r)) continue;
            err = cudaMemsetAsync(e->cur_G[r], 0, sizeof(double) * (size_t)e->members[r]->E * e->members[r]->P * 5, bs);
          }
          for (int k = 0; k < e->rk.stages && err == cudaSuccess; ++k)
            err = u.r >= 0 ? one_member_stage(e, u.r, k, e->rk.A, e->rk.B, bs) : enqueue_stage(e, g, k, bs);
        }
        cudaEvent_t join;
        if (err == cudaSuccess && (err = event(&join)) == cudaSuccess && (err = cudaEventRecord(join, bs)) == cudaSuccess)
          err = cudaStreamWaitEvent(cs, join, 0);
      }
      if (err == cudaSuccess) {
        k_ens_clock_advance<<<(n + 127) / 128, 128, 0, cs>>>(e->d_clocks, n);
        err = cudaGetLastError();
      }
    }
    cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
    if (err == cudaSuccess) err = e2;
    if (err == cudaSuccess) err = cudaGraphInstantiate(&e->graph, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
    cudaStreamDestroy(cs);
    if (err != cudaSuccess) { e->graph = nullptr; return ens_fail(e, DG_ECUDA, "ensemble graph capture", err); }
    e->graph_nsteps = nsteps;
    e->graph_fv = fv_now;
  }
  ENS_CUDA(cudaGraphLaunch(e->graph, s), e, "ensemble graph launch");
  char msg[160];
  if (bounds_failed(s, msg, sizeof msg)) return ens_fail(e, DG_ECUDA, msg);   // checked builds only
  return DG_OK;
}

dg_status dg_ensemble_plan(const dg_ensemble* e, char* buf, size_t len) {
  if (!e || !buf || len == 0) return DG_EINVAL;
  std::snprintf(buf, len, "%s", e->plan_json.c_str());
  return e->plan_json.size() < len ? DG_OK : DG_EINVAL;
}

const char* dg_ensemble_last_error(const dg_ensemble* e) { return e ? e->err.c_str() : "null ensemble"; }

}  // extern "C"
