// C ABI of the HLBM library: context, device upload, the per-coarse-step
// launch schedule (level recursion, sub-cycling, CUDA graphs) and readback.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "hlbm_device.h"
#include "hlbm_internal.h"

using namespace hlbm;

namespace {
// NVTX range for the profilers' timelines (a no-op unless a tool is attached).
// With CUDA graphs the per-family ranges mark the capture at create; with
// plain launches (options.use_graphs = 0) they bracket every launch of a step.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};
}  // namespace

struct hlbm_ctx {
    Plan plan;
    DevCtx dev;
    cudaStream_t stream = nullptr;    // caller's stream
    cudaStream_t cap_stream = nullptr;  // private stream used for graph capture
    // second branch of the step: a level's boundary-ring kernel runs beside the
    // reads of its interior that follow, where the plan shows them disjoint
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool side_ok[hlbm::kMaxLevels] = {};
    // third branch: a finest step's finite-volume sub-steps run on mesh_side
    // beside the coarser levels' lattice work that follows them, until the
    // next read of the mesh state joins them back (mesh_pending)
    cudaStream_t mesh_side = nullptr;
    cudaEvent_t ev_mfork = nullptr, ev_mjoin = nullptr;
    bool mesh_pending = false;
    int fv_variant_opt = 0;
    // mass monitoring (level 0, FP64): reference mass at create, last drift
    double *mass_buf = nullptr;  // [ny0 + 1]: row sums, total
    double mass0 = 0.0, mass_drift = 0.0, mass_nodes = 0.0;
    double fv_tune_us[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    double create_ms[3] = {0.0, 0.0, 0.0};  // host set-up tables, device build, graph capture
    double build_ms[2] = {0.0, 0.0};         // device build: tables and uploads; initial state and autotuner
    AdjTables adj;                            // finite-volume adjoint tables (built on first use)
    hlbm_ctx *shadow = nullptr;               // FP32 contexts: FP64 twin holding the adjoint's tables
    struct AdjRecorder *rec = nullptr;        // set while the adjoint records a coarse step
    void *(*alloc_fn)(size_t, void *) = nullptr;
    void (*free_fn)(void *, void *) = nullptr;
    void *alloc_ctx = nullptr;
    std::vector<void *> blocks;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    // two coarse steps from each parity in one graph: the second step's
    // coarse-level lattice work runs beside the first step's last
    // finite-volume sub-steps and forces
    cudaGraphExec_t graph2[2] = {nullptr, nullptr};
    cudaGraph_t graph_tmpl[2] = {nullptr, nullptr};  // the captured graphs (child graphs of a batch)
    bool use_graphs = false;
    long steps = 0;
    long stats_base = 0;  // coarse step at which the wall-coefficient sums were last cleared
    long forces_read = 0;
    long launches = 0;            // kernels enqueued by the scheduler (counter)
    long launches_per_step = 0;   // kernels of one coarse step
    bool timing_dirty = false;    // hlbm_time_kernel ran kernels outside the schedule
    int check_every = 0;
    double *d_out = nullptr;  // fields / populations scratch, 12 doubles per node of the largest grid
    size_t d_out_n = 0;
    std::string err;
};

// A batch: independent contexts advanced by one graph launch per coarse step.
struct hlbm_batch {
    std::vector<hlbm_ctx *> ctx;
    std::vector<long> base;            // each context's step count when the batch was made
    std::vector<cudaEvent_t> ready;    // per context: its stream's pending work
    cudaEvent_t done = nullptr;        // the batch stream's work
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    long steps = 0;
    std::string err;
};

namespace {

// relative change of the total mass that the health check treats as unstable
constexpr double kMassDriftLimit = 1e-2;

thread_local std::string g_create_err;

struct CudaError {
    std::string msg;
};

void ck(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) throw CudaError{std::string(what) + ": " + cudaGetErrorString(e)};
}

void *dalloc(hlbm_ctx *c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (c->alloc_fn) {
        p = c->alloc_fn(bytes, c->alloc_ctx);
        if (!p) throw CudaError{"device allocation failed (callback)"};
    } else {
        ck(cudaMalloc(&p, bytes), "cudaMalloc");
    }
    c->blocks.push_back(p);
    return p;
}

// Frees one block of dalloc before the context ends (per-call scratch).
void dfree(hlbm_ctx *c, void *p)
{
    if (!p) return;
    auto it = std::find(c->blocks.begin(), c->blocks.end(), p);
    if (it == c->blocks.end()) return;
    c->blocks.erase(it);
    if (c->free_fn) c->free_fn(p, c->alloc_ctx);
    else cudaFree(p);
}

template <typename V> V *upload(hlbm_ctx *c, const std::vector<V> &h)
{
    V *d = (V *)dalloc(c, h.size() * sizeof(V));
    if (!h.empty()) ck(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice, c->stream), "upload");
    return d;
}

template <typename T> std::vector<T> convert(const std::vector<double> &v) { return std::vector<T>(v.begin(), v.end()); }

// Runtime parities for the start of coarse step k: level 0 alternates, finer
// levels take an even number of steps per coarse step, and the mesh buffer
// flips once per finite-volume sub-step.
void set_phase(hlbm_ctx *c, long k)
{
    DevCtx &D = c->dev;
    D.lv[0].parity = int(k & 1);
    for (int l = 1; l < D.L; l++) D.lv[l].parity = 0;
    long per = long(D.n_sub + (D.fv_filter > 0.0 ? 1 : 0)) << (D.L - 1);
    D.m.gcur = int((k * per) & 1);
    for (int l = 0; l < D.L; l++) {  // steps of level l done before coarse step k: k 2^l
        DevLevel &dl = D.lv[l];
        if (!dl.snap[0]) continue;
        dl.spar = int((k << l) & 1);
        dl.snapA = dl.snap[dl.spar];
        dl.snapB = dl.snap[dl.spar ^ 1];
    }
    D.m.qpar = int((k << (D.L - 1)) & 1);  // finest steps done before coarse step k
    D.m.Q0 = D.m.Qb[D.m.qpar];
    D.m.Q1 = D.m.Qb[D.m.qpar ^ 1];
}

template <typename T, typename S> void advance(hlbm_ctx *c, int lvl, double theta, cudaStream_t s);

// What the adjoint of a coarse step needs from its forward pass, per level
// step (in schedule order): the level's lattice at the step start and after
// its boundary ring was written, the child's lattice when the restriction
// reads it, the parent band data the prolongation read, and (finest level
// with a mesh) the mesh state and interface data.  Copies on the stream,
// into blocks freed by release().
}  // namespace

struct LevelRec {
    int l = 0, P = 0;
    double theta = 0.0;
    double *f_start = nullptr, *f_end = nullptr, *f_child = nullptr, *sA = nullptr, *sB = nullptr;
    double *g_start = nullptr, *Q0 = nullptr, *Q1 = nullptr;
};
struct AdjRecorder {
    hlbm_ctx *c = nullptr;
    cudaStream_t s = nullptr;
    bool f32 = false;  // the recorded buffers hold FP32 values (widened to FP64 when kept)
    std::vector<LevelRec> recs;
    std::vector<void *> blocks;
    double *keep(const void *src, size_t doubles);
    void release();
};
namespace {
void dfree(hlbm_ctx *c, void *p);
void *dalloc(hlbm_ctx *c, size_t bytes);
}  // namespace
double *AdjRecorder::keep(const void *src, size_t doubles)
{
    double *p = (double *)dalloc(c, doubles * sizeof(double));
    blocks.push_back(p);
    if (f32) launch_widen((const float *)src, p, doubles, s);
    else ck(cudaMemcpyAsync(p, src, doubles * sizeof(double), cudaMemcpyDeviceToDevice, s), "record");
    return p;
}
void AdjRecorder::release()
{
    for (void *p : blocks) dfree(c, p);
    blocks.clear();
    recs.clear();
}

namespace {

const char *const kLatticeRange[kMaxLevels] = {"lattice: level 0", "lattice: level 1", "lattice: level 2",
                                               "lattice: level 3", "lattice: level 4", "lattice: level 5",
                                               "lattice: level 6", "lattice: level 7"};

// One step of level lvl on its own clock; theta: parent-time fraction at the
// end of the step (refills the boundary ring by prolongation).
// Branch of the step graph: work enqueued on c->side between fork and join
// runs beside the work enqueued on s in between.
void fork(hlbm_ctx *c, cudaStream_t s)
{
    ck(cudaEventRecord(c->ev_fork, s), "event record");
    ck(cudaStreamWaitEvent(c->side, c->ev_fork, 0), "stream wait");
}
void join(hlbm_ctx *c, cudaStream_t s)
{
    ck(cudaEventRecord(c->ev_join, c->side), "event record");
    ck(cudaStreamWaitEvent(s, c->ev_join, 0), "stream wait");
}
// The mesh branch: the finite-volume sub-steps of a finest step (they read
// and write only the mesh state and read the Eq. 9 ring data) leave s on
// c->mesh_side; s continues with the coarser levels' lattice work (which
// touches neither), and every later reader or writer of the mesh state or of
// the ring data (the next hole and ring interpolations, the forces, an
// adjoint record) joins the branch first.
void mesh_fork(hlbm_ctx *c, cudaStream_t s)
{
    ck(cudaEventRecord(c->ev_mfork, s), "event record");
    ck(cudaStreamWaitEvent(c->mesh_side, c->ev_mfork, 0), "stream wait");
    c->mesh_pending = true;
}
void mesh_join(hlbm_ctx *c, cudaStream_t s)
{
    if (!c->mesh_pending) return;
    ck(cudaEventRecord(c->ev_mjoin, c->mesh_side), "event record");
    ck(cudaStreamWaitEvent(s, c->ev_mjoin, 0), "stream wait");
    c->mesh_pending = false;
}

template <typename T, typename S> void level_step(hlbm_ctx *c, int lvl, double theta, cudaStream_t s)
{
    DevCtx &D = c->dev;
    bool hybrid = (lvl == D.L - 1) && D.m.n > 0;
    bool child = lvl < D.L - 1;
    if (hybrid) mesh_join(c, s);  // the previous finest step's sub-steps
    if (c->rec) {
        AdjRecorder &R = *c->rec;
        LevelRec r;
        r.l = lvl;
        r.P = D.lv[lvl].parity;
        r.theta = theta;
        r.f_start = R.keep(D.lv[lvl].f, 9 * D.lv[lvl].stride);
        if (hybrid) {
            r.g_start = R.keep(D.m.g[D.m.gcur], size_t(9) * D.m.Np);
            r.Q0 = R.keep(D.m.Q0, 12 * size_t(std::max(1, D.m.n_ring)));
        }
        R.recs.push_back(r);
    }
    if (hybrid) {
        // Eq. 9 data at t: already in Q0 (the previous step's data at t + 1,
        // or the initial state's)
        Range r("overlap: hole interpolation");
        launch_hole_interp<T, S>(D, s);  // Eq. 4: post-collision of the hole boundary
        c->launches += (D.m.n_is > 0);
    }
    {
        Range r(kLatticeRange[lvl]);
        launch_collide<T, S>(D, lvl, s);  // Eq. 1
    }
    D.lv[lvl].parity ^= 1;
    // The level's boundary ring (outer conditions / prolongation) is written
    // beside what reads the level's interior next: the child's band snapshot
    // (joined in advance) or the ring data of the mesh (joined here).
    const bool branch = c->side_ok[lvl] && (child || hybrid);
    cudaStream_t sb = s;
    if (branch) {
        fork(c, s);
        sb = c->side;
    }
    {
        Range r(lvl == 0 ? "lattice: outer conditions" : "refine: prolongation");
        if (lvl == 0) launch_outer_bc<T, S>(D, sb);
        else launch_prolong<T, S>(D, lvl, theta, sb);
    }
    c->launches += 2;
    if (c->rec) {
        AdjRecorder &R = *c->rec;
        LevelRec &r = R.recs.back();
        r.f_end = R.keep(D.lv[lvl].f, 9 * D.lv[lvl].stride);
        if (lvl > 0) {
            const DevLevel &pl = D.lv[lvl - 1];
            r.sA = R.keep(pl.snapA, 12 * size_t(pl.band_n));
            r.sB = R.keep(pl.snapB, 12 * size_t(pl.band_n));
        }
    }
    if (hybrid) {
        {
            Range r("overlap: ring interpolation");
            launch_ring_interp<T, S>(D, true, s);  // Eq. 9 data at t + 1, ring state of sub-step 0
        }
        if (c->rec) c->rec->recs.back().Q1 = c->rec->keep(D.m.Q1, 12 * size_t(std::max(1, D.m.n_ring)));
        if (branch) join(c, s);
        Range r("fv: sub-steps");
        cudaStream_t sm = s;
        if (c->mesh_side && !c->rec) {
            mesh_fork(c, s);
            sm = c->mesh_side;
        }
        for (int m = 0; m < D.n_sub; m++) {  // Eq. 3, Eq. 5-7, wall rule
            launch_fv<T, S>(D, m, sm);
            D.m.gcur ^= 1;
        }
        c->launches += 1 + D.n_sub;
        if (D.fv_filter > 0.0) {  // optional odd-even filter of the mesh state
            launch_fv_filter<T, S>(D, sm);
            D.m.gcur ^= 1;
            c->launches += 2;
        }
        D.m.qpar ^= 1;  // the data at t + 1 is the next step's data at t
        std::swap(D.m.Q0, D.m.Q1);
    }
}

template <typename T, typename S> void advance(hlbm_ctx *c, int lvl, double theta, cudaStream_t s)
{
    DevCtx &D = c->dev;
    bool child = lvl < D.L - 1;
    // the band at the start of the step (snapA) is the previous step's snapB
    // (or the initial state's)
    level_step<T, S>(c, lvl, theta, s);
    if (child) {
        {
            Range r("refine: band snapshot");
            launch_snapshot<T, S>(D, lvl, true, s);
        }
        if (c->side_ok[lvl]) join(c, s);
        advance<T, S>(c, lvl + 1, 0.5, s);
        advance<T, S>(c, lvl + 1, 1.0, s);
        if (c->rec) {  // the child's lattice as the restriction reads it
            AdjRecorder &R = *c->rec;
            for (size_t k = R.recs.size(); k-- > 0;)
                if (R.recs[k].l == lvl) {
                    R.recs[k].f_child = R.keep(D.lv[lvl + 1].f, 9 * D.lv[lvl + 1].stride);
                    break;
                }
        }
        Range r("refine: restriction");
        launch_restrict<T, S>(D, lvl, s);
        c->launches += 2;
        DevLevel &dl = D.lv[lvl];
        dl.spar ^= 1;
        std::swap(dl.snapA, dl.snapB);
    }
}

// One coarse step on s.  keep_branch: another coarse step follows in the same
// graph, so the forces (which read the mesh state) stay on the mesh branch
// and the next step's lattice work need not wait for them.
template <typename T, typename S> void coarse_step(hlbm_ctx *c, cudaStream_t s, bool keep_branch = false)
{
    long before = c->launches;
    Range step("coarse step");
    advance<T, S>(c, 0, 0.0, s);
    cudaStream_t sf = s;
    if (keep_branch && c->mesh_pending) sf = c->mesh_side;
    else mesh_join(c, s);
    if (c->dev.m.n > 0) {
        Range r("forces");
        launch_forces<T, S>(c->dev, sf);
        c->launches += 2;
        if (c->dev.m.wall_stats) {
            launch_wall_stats<T, S>(c->dev, sf);
            c->launches += 1;
        }
    }
    c->launches_per_step = c->launches - before;
}

void enqueue_coarse_step(hlbm_ctx *c, cudaStream_t s, bool keep_branch = false)
{
    if (c->plan.precision == HLBM_FP32) coarse_step<float, float>(c, s, keep_branch);
    else if (c->plan.precision == HLBM_FP16S) coarse_step<float, __half>(c, s, keep_branch);
    else coarse_step<double, double>(c, s, keep_branch);
}

// Total mass of level 0 now (FP64; synchronises the context's stream).
double level0_mass(hlbm_ctx *c)
{
    const int ny = c->dev.lv[0].ny;
    if (c->plan.precision == HLBM_FP32) launch_mass<float, float>(c->dev, c->mass_buf, c->mass_buf + ny, c->stream);
    else if (c->plan.precision == HLBM_FP16S)
        launch_mass<float, __half>(c->dev, c->mass_buf, c->mass_buf + ny, c->stream);
    else launch_mass<double, double>(c->dev, c->mass_buf, c->mass_buf + ny, c->stream);
    ck(cudaGetLastError(), "mass kernel");
    double dev = 0.0;
    ck(cudaMemcpyAsync(&dev, c->mass_buf + ny, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "D2H");
    ck(cudaStreamSynchronize(c->stream), "sync");
    return c->mass_nodes + dev;
}

template <typename T, typename S> void init_state(hlbm_ctx *c)
{
    DevCtx &D = c->dev;
    const Plan &P = c->plan;
    cudaStream_t s = c->stream;
    for (int l = 0; l < D.L; l++) {
        D.lv[l].parity = 0;
        launch_init_level<T, S>(D, l, P.seed, P.perturb, s);
    }
    // make the initial state consistent across the interfaces
    launch_outer_bc<T, S>(D, s);
    for (int l = 1; l < D.L; l++) {
        launch_snapshot<T, S>(D, l - 1, false, s);
        launch_snapshot<T, S>(D, l - 1, true, s);
        launch_prolong<T, S>(D, l, 0.0, s);
    }
    for (int l = D.L - 2; l >= 0; l--) launch_restrict<T, S>(D, l, s);
    if (D.m.n > 0) {
        // mesh: rho = 1 + perturb xi, u = (u0, 0) (0 on wall nodes), f^neq = 0;
        // planes (rho - 1, ux, uy, f^neq_3..8), device order
        std::vector<T> g(size_t(9) * D.m.Np, T(0));
        for (int p = 0; p < P.n; p++) {
            int q = P.inv[p];
            g[q] = T(P.perturb * init_deviate(P.seed, kMeshGrid, uint64_t(p)));
            g[size_t(D.m.Np) + q] = T(P.kind[p] == HLBM_NODE_WALL ? 0.0 : P.u0);
        }
        ck(cudaMemcpyAsync(D.m.g[0], g.data(), g.size() * sizeof(T), cudaMemcpyHostToDevice, s), "upload mesh state");
        ck(cudaStreamSynchronize(s), "sync");  // g (host) goes out of scope
        D.m.gcur = 0;
        launch_ring_interp<T, S>(D, false, s);  // Q0
        launch_ring_interp<T, S>(D, true, s);   // Q1 and the ring state at theta = 0
    }
    ck(cudaGetLastError(), "init kernels");
}

// One tiling of the finite-volume sub-step kernel (tiles of `rows` device
// rows): each tile's staged list and the operator entries with their
// positions in it, in a per-slice order spread over the shared-memory banks;
// uploads them into tl (tl.rows stays 0 if a tile's staging does not fit in
// shared memory).
template <typename T>
void build_tiles(hlbm_ctx *c, const std::vector<int> &odp, const std::vector<int> &od, const std::vector<int> &sptr,
                 const std::vector<int> &slen, int rows, FvTiles &tl)
{
    const Plan &P = c->plan;
    const DevMesh &M = c->dev.m;
    using E = typename std::conditional<std::is_same<T, float>::value, float4, double4_32a>::type;
    tl = FvTiles();
    const int n_tiles = (P.n + rows - 1) / rows;
    int max_halo = 0;
    std::vector<int> hptr(n_tiles + 1, 0), hnodes;
    // tile t's staged list: its own device rows r0 .. r0 + rows - 1 (the last
    // tile's run reaches into the padding rows, never referenced), which the
    // kernel copies in bulk, then the other nodes its rows touch, sorted,
    // which it gathers; an entry's column is its node's position in the list
    std::vector<std::vector<int>> halo(n_tiles);
    parallel_for(n_tiles, [&](int t0, int t1) {
        for (int t = t0; t < t1; t++) {
            const int r0 = t * rows;
            std::vector<int> &h = halo[t];
            for (int r = r0; r < std::min(P.n, r0 + rows); r++)
                for (int j = odp[r]; j < odp[r + 1]; j++) {
                    const int c = P.inv[P.col[od[j]]];
                    if (c < r0 || c >= r0 + rows) h.push_back(c);
                }
            std::sort(h.begin(), h.end());
            h.erase(std::unique(h.begin(), h.end()), h.end());
            std::vector<int> own(rows);
            for (int j = 0; j < rows; j++) own[j] = r0 + j;
            h.insert(h.begin(), own.begin(), own.end());
        }
    }, 16);
    for (int t = 0; t < n_tiles; t++) {
        hptr[t + 1] = hptr[t] + int(halo[t].size());
        max_halo = std::max(max_halo, int(halo[t].size()));
    }
    hnodes.resize(hptr[n_tiles]);
    parallel_for(n_tiles, [&](int t0, int t1) {
        for (int t = t0; t < t1; t++) std::copy(halo[t].begin(), halo[t].end(), hnodes.begin() + hptr[t]);
    }, 16);
    halo.clear();
    // position of device node c in tile t's staged list
    auto halo_pos = [&](int t, int c) {
        const int r0 = t * rows;
        if (c >= r0 && c < r0 + rows) return c - r0;
        const int *h0 = hnodes.data() + hptr[t] + rows, *h1 = hnodes.data() + hptr[t + 1];
        return rows + int(std::lower_bound(h0, h1, c) - h0);
    };
    std::vector<E> ent;
    auto set_col = [](E &v, int col) {
        if (std::is_same<T, float>::value) { float fcol; std::memcpy(&fcol, &col, 4); std::memcpy(&v.w, &fcol, 4); }
        else v.w = T(col);
    };
    // entries carry dt s_Pk and (dt / tau_u) C_Pk (the sub-step's constants folded in)
    const double dt = P.n_sub > 0 ? 1.0 / P.n_sub : 0.0, dt_tau = dt / P.tau_u;
    ent.resize(size_t(sptr[M.n_slices]));
    // Entry order within a row is free (the sums are over all of them), so
    // each slice orders its 32 rows' entries slot by slot to spread the 32
    // shared-memory reads of one slot over the banks: a row takes, among its
    // remaining neighbours, one whose staged position another row of the
    // slice already reads in this slot (a broadcast), else one in the bank
    // with the fewest distinct positions so far (lowest entry on ties);
    // padding entries (zero coefficients) read a position already read.
    parallel_for(M.n_slices, [&](int sl0, int sl1) {
        std::vector<int> pos[32], order[32];
        std::vector<int> stamp(size_t(max_halo) + 1, -1);  // slot stamp of each staged position
        int stamp_id = 0;
        for (int sl = sl0; sl < sl1; sl++) {
            const int len = slen[sl];
            const size_t base = size_t(sptr[sl]);
            uint32_t used[32];
            for (int l = 0; l < 32; l++) {
                const int r = sl * 32 + l;
                pos[l].clear();
                order[l].clear();
                used[l] = 0;
                if (r >= P.n) continue;
                for (int j = odp[r]; j < odp[r + 1]; j++) pos[l].push_back(halo_pos(r / rows, P.inv[P.col[od[j]]]));
            }
            bool small = true;  // the bank-aware order tracks up to 32 entries per row
            for (int l = 0; l < 32; l++) small = small && pos[l].size() <= 32;
            if (!small)
                for (int l = 0; l < 32; l++)
                    for (int j = 0; j < int(pos[l].size()); j++) order[l].push_back(j);
            for (int e = 0; e < len; e++) {
                const int sid = stamp_id++;
                if (!small) {
                    for (int l = 0; l < 32; l++) {
                        const int r = sl * 32 + l;
                        E v{};
                        if (e < int(order[l].size())) {
                            const int j = order[l][e], k = od[odp[r] + j];
                            v.x = T(dt * P.sx[k]); v.y = T(dt * P.sy[k]); v.z = T(dt_tau * P.cc[k]);
                            set_col(v, pos[l][j]);
                        } else {
                            v.x = v.y = v.z = T(0);
                            set_col(v, 0);
                        }
                        ent[base + size_t(32) * e + l] = v;
                    }
                    continue;
                }
                int bank_n[32] = {0}, first = -1;
                for (int l = 0; l < 32; l++) {
                    const int nr = int(pos[l].size());
                    int best = -1, best_cost = 1 << 30;
                    for (int j = 0; j < nr && j < 32; j++) {
                        if (used[l] >> j & 1u) continue;
                        const int k = pos[l][j];
                        const int cost = stamp[k] == sid ? -1 : bank_n[k & 31];
                        if (cost < best_cost) { best_cost = cost; best = j; }
                    }
                    if (best >= 0) {
                        used[l] |= 1u << best;
                        order[l].push_back(best);
                        const int k = pos[l][best];
                        if (stamp[k] != sid) {
                            stamp[k] = sid;
                            bank_n[k & 31]++;
                            if (first < 0) first = k;
                        }
                    }
                }
                const int pad_col = first < 0 ? 0 : first;
                for (int l = 0; l < 32; l++) {
                    const int r = sl * 32 + l;
                    E v{};
                    if (e < int(order[l].size())) {
                        const int j = order[l][e], k = od[odp[r] + j];
                        v.x = T(dt * P.sx[k]); v.y = T(dt * P.sy[k]); v.z = T(dt_tau * P.cc[k]);
                        set_col(v, pos[l][j]);
                    } else {
                        v.x = v.y = v.z = T(0);  // padding: zero coefficients on a position already read
                        set_col(v, pad_col);
                    }
                    ent[base + size_t(32) * e + l] = v;
                }
            }
        }
    }, 64);
    int max_tile_ent = 0;
    for (int t = 0; t < n_tiles; t++)
        max_tile_ent = std::max(max_tile_ent, sptr[std::min(M.n_slices, (rows / 32) * (t + 1))] - sptr[(rows / 32) * t]);
    // mbarriers (16 B), the tile's entries, the staged states (planes of a
    // stride rounded up to 4 values: 16-byte aligned bulk copies)
    const size_t smem = 16 + size_t(max_tile_ent) * sizeof(E) + size_t((max_halo + 3) & ~3) * 9 * sizeof(T);
    if (smem > 200 * 1024) return;
    tl.rows = rows;
    tl.n_tiles = n_tiles;
    tl.max_tile_ent = max_tile_ent;
    tl.max_halo = max_halo;
    tl.smem_bytes = smem;
    configure_fv<T, T>(tl);
    configure_fv_prefetch<T, T>(tl);
    tl.halo_ptr = upload(c, hptr);
    tl.halo_nodes = upload(c, hnodes);
    tl.ent = upload(c, ent);
}

template <typename T> void upload_mesh(hlbm_ctx *c)
{
    Plan &P = c->plan;
    DevMesh &M = c->dev.m;
    const LevelPlan &F = P.lv[P.L - 1];
    const DevLevel &FL = c->dev.lv[P.L - 1];
    M.n = P.n;
    // rows padded to whole tiles of either tiling: the sub-step kernel copies
    // every tile's rows in bulk
    M.Np = (P.n + kTileRowsWide - 1) / kTileRowsWide * kTileRowsWide;
    M.n_wall = P.n_wall;
    M.ring_start = P.ring_start;
    M.n_ring = P.n_ring;
    for (int b = 0; b < 2; b++) M.g[b] = dalloc(c, size_t(9) * M.Np * sizeof(T));
    if (c->dev.fv_filter > 0.0) M.lap = dalloc(c, size_t(9) * M.Np * sizeof(T));
    // the self entry of a row is not stored: its streaming term vanishes in the
    // difference form and its collision weight is C_PP = 11/18 on every node;
    // off-diagonal entries of device row r: od[odp[r] .. odp[r + 1])
    std::vector<int> odp(size_t(P.n) + 1, 0), od;
    od.reserve(P.col.size());
    for (int r = 0; r < P.n; r++) {
        const int old = P.perm[r];
        for (int k = P.rowptr[old]; k < P.rowptr[old + 1]; k++)
            if (P.col[k] != old) od.push_back(k);
        odp[r + 1] = int(od.size());
    }
    // sliced-ELL operator rows in device order, 32-row slices: lengths and
    // offsets (the same for every tiling), then each tiling's entries
    M.n_slices = M.Np / 32;
    std::vector<int> sptr(size_t(M.n_slices) + 1), slen(M.n_slices);
    size_t n_ent = 0;
    for (int sl = 0; sl < M.n_slices; sl++) {
        int len = 0;
        for (int l = 0; l < 32; l++) {
            int r = sl * 32 + l;
            if (r < P.n) len = std::max(len, odp[r + 1] - odp[r]);
        }
        sptr[sl] = int(n_ent);
        slen[sl] = len;
        n_ent += size_t(32) * len;
    }
    sptr[M.n_slices] = int(n_ent);
    build_tiles<T>(c, odp, od, sptr, slen, kTileRows, M.tl);
    if (!M.tl.rows) throw CudaError{"mesh tiles touch too many nodes for shared memory"};
    // FP32: also the wide tiling, when a variant of it is asked for or, for
    // the autotuner, when the 128-row tiles need more than two waves of
    // resident blocks (8 per SM): only there did the wide tiles win (the
    // 1.5 M-node mesh, ~10 waves; not the 200 k mesh, 1.3 waves)
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 0;
    }
    const bool many_waves = sms > 0 && M.tl.n_tiles > 2 * 8 * sms;
    if (std::is_same<T, float>::value && (c->fv_variant_opt > 4 || (c->fv_variant_opt == 0 && many_waves)))
        build_tiles<T>(c, odp, od, sptr, slen, kTileRowsWide, M.tl_alt);
    M.slice_ptr = upload(c, sptr);
    M.slice_len = upload(c, slen);
    M.Qb[0] = dalloc(c, size_t(12) * std::max(1, P.n_ring) * sizeof(T));
    M.Qb[1] = dalloc(c, size_t(12) * std::max(1, P.n_ring) * sizeof(T));
    M.qpar = 0;
    M.Q0 = M.Qb[0];
    M.Q1 = M.Qb[1];
    // Eq. 8 stencils
    M.n_is = int(P.is_node.size());
    std::vector<int> isn(M.n_is), isd(6 * size_t(M.n_is));
    for (int s = 0; s < M.n_is; s++) {
        int x = P.is_node[s] % F.nx, y = P.is_node[s] / F.nx;
        isn[s] = (y + 1) * FL.pitch + x + 1;
        for (int k = 0; k < 6; k++) isd[6 * s + k] = P.inv[P.is_don[6 * s + k]];
    }
    M.is_n = upload(c, isn);
    M.is_don = upload(c, isd);
    M.is_w = upload(c, convert<T>(P.is_w));
    // Eq. 9 stencils
    std::vector<int> rd(9 * size_t(P.n_ring));
    for (size_t k = 0; k < rd.size(); k++) {
        int x = P.ring_don[k] % F.nx, y = P.ring_don[k] / F.nx;
        rd[k] = (y + 1) * FL.pitch + x + 1;
    }
    M.ring_don = upload(c, rd);
    M.ring_w = upload(c, convert<T>(P.ring_w));
    // wall edges: device-order nodes and the normal times length into the fluid
    M.n_edges = int(P.wea.size());
    std::vector<int> ea(M.n_edges), eb(M.n_edges);
    std::vector<double> wn(2 * size_t(M.n_edges));
    for (int e = 0; e < M.n_edges; e++) {
        ea[e] = P.inv[P.wea[e]];
        eb[e] = P.inv[P.web[e]];
        double dx = P.xy[2 * P.web[e]] - P.xy[2 * P.wea[e]], dy = P.xy[2 * P.web[e] + 1] - P.xy[2 * P.wea[e] + 1];
        wn[2 * e] = -dy;  // left normal: from the body into the fluid
        wn[2 * e + 1] = dx;
    }
    M.wea = upload(c, ea);
    M.web = upload(c, eb);
    M.wn = upload(c, wn);
    M.inv = upload(c, P.inv);
    if (M.wall_stats && P.n_wall > 0) {
        std::vector<double> ns(4 * size_t(P.n_wall));
        for (int w = 0; w < P.n_wall; w++)
            for (int k = 0; k < 4; k++) ns[4 * size_t(w) + k] = P.wall_geo[7 * size_t(w) + 3 + k];
        M.wall_ns = upload(c, ns);
        M.wall_acc = (double *)dalloc(c, 3 * size_t(P.n_wall) * sizeof(double));
        ck(cudaMemsetAsync(M.wall_acc, 0, 3 * size_t(P.n_wall) * sizeof(double), c->stream), "memset");
    }
}

template <typename T, typename S> void build_device(hlbm_ctx *c)
{
    Plan &P = c->plan;
    DevCtx &D = c->dev;
    D.L = P.L;
    D.u0 = P.u0;
    D.tau_u = P.tau_u;
    D.n_sub = P.n_sub;
    D.dt_u = P.n_sub > 0 ? 1.0 / P.n_sub : 0.0;
    D.qdyn = P.qdyn;
    const auto t_beg = std::chrono::steady_clock::now();
    // FP16S storage shift: the free-stream equilibrium minus the weights
    {
        static const double W[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
        static const int CXh[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
        for (int i = 0; i < 9; i++) {
            double cu = CXh[i] * P.u0;
            D.shift.s[i] = float(W[i] * (3.0 * cu + 4.5 * cu * cu - 1.5 * P.u0 * P.u0));
        }
    }
    size_t maxnodes = size_t(std::max(P.n, 1));
    for (int l = 0; l < P.L; l++) {
        const LevelPlan &lp = P.lv[l];
        DevLevel &dl = D.lv[l];
        dl.nx = lp.nx;
        dl.ny = lp.ny;
        dl.pitch = (lp.nx + 2 + 31) / 32 * 32;
        dl.stride = size_t(lp.ny + 2) * dl.pitch;
        dl.f = dalloc(c, 9 * dl.stride * sizeof(S));
        dl.tau = lp.tau;
        if (!lp.hx0.empty()) {
            dl.hx0 = upload(c, lp.hx0);
            dl.hx1 = upload(c, lp.hx1);
        }
        dl.has_child = lp.has_child;
        if (lp.has_child) {
            dl.cox = lp.cox; dl.coy = lp.coy; dl.cmx = lp.cmx; dl.cmy = lp.cmy;
            dl.band_n = 2 * (lp.cmx + 2) + 2 * (lp.cmy + 2);
            dl.snap[0] = dl.snapA = dalloc(c, size_t(12) * dl.band_n * sizeof(T));
            dl.snap[1] = dl.snapB = dalloc(c, size_t(12) * dl.band_n * sizeof(T));
            dl.spar = 0;
        }
        maxnodes = std::max(maxnodes, size_t(lp.nx) * lp.ny);
    }
    if (P.n > 0) upload_mesh<T>(c);
    D.force_cap = std::max(1, D.force_cap);
    D.force_buf = (double *)dalloc(c, size_t(2) * D.force_cap * sizeof(double));
    D.force_partial = (double *)dalloc(c, size_t(2) * std::max(1, (D.m.n_edges + 127) / 128) * sizeof(double));
    D.force_counter = (int *)dalloc(c, 2 * sizeof(int));
    D.flag = D.force_counter + 1;
    ck(cudaMemsetAsync(D.force_counter, 0, 2 * sizeof(int), c->stream), "memset");
    c->d_out_n = maxnodes;
    c->d_out = (double *)dalloc(c, maxnodes * 12 * sizeof(double));
    c->mass_buf = (double *)dalloc(c, (size_t(D.lv[0].ny) + 1) * sizeof(double));
    {
        const LevelPlan &l0 = P.lv[0];
        double nodes = double(l0.nx) * l0.ny;
        for (size_t y = 0; y < l0.hx0.size(); y++) nodes -= double(l0.hx1[y] - l0.hx0[y]);
        c->mass_nodes = nodes;
    }
    const auto t_up = std::chrono::steady_clock::now();
    init_state<T, S>(c);
    if (P.n > 0) {
        DevMesh &M = D.m;
        if (c->plan.precision == HLBM_FP64) {
            M.fv_variant = 1;
        } else if (c->fv_variant_opt > 4) {  // a variant of the wide tiling, if it was built
            if (!M.tl_alt.rows) throw CudaError{"fv_variant 5..8: the wide tiling does not fit in shared memory"};
            std::swap(M.tl, M.tl_alt);
            M.fv_variant = c->fv_variant_opt - 4;
        } else if (c->fv_variant_opt > 0) {
            M.fv_variant = c->fv_variant_opt;
        } else {
            fv_autotune<T, S>(D, c->stream, c->fv_tune_us);
        }
        ck(cudaStreamSynchronize(c->stream), "sync");
        // the tiling not kept
        dfree(c, M.tl_alt.ent);
        dfree(c, M.tl_alt.halo_ptr);
        dfree(c, M.tl_alt.halo_nodes);
        M.tl_alt = FvTiles();
        ck(cudaGetLastError(), "finite-volume autotuner");
    }
    ck(cudaStreamSynchronize(c->stream), "sync");
    const auto t_end = std::chrono::steady_clock::now();
    c->build_ms[0] = std::chrono::duration<double, std::milli>(t_up - t_beg).count();
    c->build_ms[1] = std::chrono::duration<double, std::milli>(t_end - t_up).count();
}

void capture_graphs(hlbm_ctx *c)
{
    ck(cudaStreamSynchronize(c->stream), "sync");
    for (int k = 0; k < 2; k++) {
        set_phase(c, k);
        cudaGraph_t g = nullptr;
        ck(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        try {
            enqueue_coarse_step(c, c->cap_stream);
        } catch (...) {
            cudaStreamEndCapture(c->cap_stream, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        ck(cudaStreamEndCapture(c->cap_stream, &g), "end capture");
        c->graph_tmpl[k] = g;
        ck(cudaGraphInstantiate(&c->graph[k], g, 0), "graph instantiate");
    }
    for (int k = 0; k < 2; k++) {  // coarse steps k, k + 1 (mod 2)
        cudaGraph_t g = nullptr;
        set_phase(c, k);
        ck(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        try {
            enqueue_coarse_step(c, c->cap_stream, true);
            set_phase(c, k + 1);
            enqueue_coarse_step(c, c->cap_stream);
        } catch (...) {
            cudaStreamEndCapture(c->cap_stream, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        ck(cudaStreamEndCapture(c->cap_stream, &g), "end capture");
        const cudaError_t e = cudaGraphInstantiate(&c->graph2[k], g, 0);
        cudaGraphDestroy(g);
        ck(e, "graph instantiate");
    }
    set_phase(c, c->steps);
}

// Where the boundary-ring kernel of a level may run beside the next reads of
// its interior.  With the in-place AA layout a node's state at odd parity sits
// in its neighbours' slots, so the written and read regions must be apart by
// a margin: a child box at least 4 nodes inside its parent (the band read
// around it, one node wider, against the ring written at the edge), and ring
// interpolation donors at least 3 nodes from the finest level's edge.
void set_branches(hlbm_ctx *c)
{
    const Plan &P = c->plan;
    for (int l = 0; l < P.L; l++) {
        const LevelPlan &lp = P.lv[l];
        bool ok = false;
        if (lp.has_child) {
            ok = lp.cox >= 4 && lp.coy >= 4 && lp.cox + lp.cmx <= lp.nx - 5 && lp.coy + lp.cmy <= lp.ny - 5;
        } else if (l == P.L - 1 && P.n > 0 && !P.ring_don.empty()) {
            ok = true;
            for (int d : P.ring_don) {
                const int x = d % lp.nx, y = d / lp.nx;
                if (x < 3 || y < 3 || x > lp.nx - 4 || y > lp.ny - 4) { ok = false; break; }
            }
        }
        c->side_ok[l] = ok;
    }
}

void release(hlbm_ctx *c)
{
    for (int k = 0; k < 2; k++) {
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
        if (c->graph2[k]) cudaGraphExecDestroy(c->graph2[k]);
        if (c->graph_tmpl[k]) cudaGraphDestroy(c->graph_tmpl[k]);
    }
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (void *p : c->blocks) {
        if (c->free_fn) c->free_fn(p, c->alloc_ctx);
        else cudaFree(p);
    }
    c->blocks.clear();
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->mesh_side) cudaStreamDestroy(c->mesh_side);
    if (c->ev_mfork) cudaEventDestroy(c->ev_mfork);
    if (c->ev_mjoin) cudaEventDestroy(c->ev_mjoin);
}

}  // namespace

void hlbm::set_thread_error(const std::string &msg) { g_create_err = msg; }

namespace {

int fail(hlbm_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    else g_create_err = msg;
    return code;
}

}  // namespace

extern "C" {

int hlbm_create(const hlbm_level *lv, int n_levels, const hlbm_mesh *m, double Re, double Ma, double aoa_deg,
                const hlbm_options *opt, hlbm_ctx **out)
{
    if (!out) return fail(nullptr, HLBM_EINVAL, "out is NULL");
    *out = nullptr;
    hlbm_ctx *c = new (std::nothrow) hlbm_ctx();
    if (!c) return fail(nullptr, HLBM_ENOMEM, "host allocation failed");
    Range create("hlbm_create");
    std::string err;
    int rc;
    auto t0 = std::chrono::steady_clock::now();
    auto lap = [&t0](double &ms) {
        const auto t1 = std::chrono::steady_clock::now();
        ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        t0 = t1;
    };
    try {
        Range r("set-up tables");
        rc = build_plan(lv, n_levels, m, Re, Ma, aoa_deg, opt, c->plan, err);
    } catch (const std::bad_alloc &) {
        delete c;
        return fail(nullptr, HLBM_ENOMEM, "host allocation failed");
    }
    lap(c->create_ms[0]);
    if (rc != HLBM_OK) { delete c; return fail(nullptr, rc, err); }
    hlbm_options o{};
    if (opt) o = *opt;
    c->stream = (cudaStream_t)o.stream;
    c->alloc_fn = o.alloc;
    c->free_fn = o.alloc ? o.free : nullptr;
    c->alloc_ctx = o.alloc_ctx;
    c->use_graphs = o.use_graphs != 0;
    c->dev.m.wall_stats = o.wall_stats != 0;
    if (o.fv_variant < 0 || o.fv_variant > 8) { delete c; return fail(nullptr, HLBM_EINVAL, "fv_variant must be in 0..8"); }
    c->fv_variant_opt = o.fv_variant;
    if (!(o.fv_filter >= 0.0 && o.fv_filter <= 1.0)) {
        delete c;
        return fail(nullptr, HLBM_EINVAL, "fv_filter must be in [0, 1]");
    }
    c->dev.fv_filter = o.fv_filter;
    c->check_every = std::max(0, o.check_every);
    c->dev.force_cap = o.force_cap > 0 ? o.force_cap : 4096;
    try {
        ck(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "stream create");
        ck(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "stream create");
        ck(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "event create");
        ck(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "event create");
        ck(cudaStreamCreateWithFlags(&c->mesh_side, cudaStreamNonBlocking), "stream create");
        ck(cudaEventCreateWithFlags(&c->ev_mfork, cudaEventDisableTiming), "event create");
        ck(cudaEventCreateWithFlags(&c->ev_mjoin, cudaEventDisableTiming), "event create");
        set_branches(c);
        {
            Range r("device upload and autotune");
            if (c->plan.precision == HLBM_FP32) build_device<float, float>(c);
            else if (c->plan.precision == HLBM_FP16S) build_device<float, __half>(c);
            else build_device<double, double>(c);
        }
        c->mass0 = level0_mass(c);
        lap(c->create_ms[1]);
        if (c->use_graphs) {
            Range r("graph capture");
            capture_graphs(c);
        }
        ck(cudaStreamSynchronize(c->stream), "sync after create");
        lap(c->create_ms[2]);
    } catch (const CudaError &e) {
        std::string msg = e.msg;
        release(c);
        delete c;
        return fail(nullptr, msg.find("alloc") != std::string::npos ? HLBM_ENOMEM : HLBM_ECUDA, msg);
    } catch (const std::bad_alloc &) {
        release(c);
        delete c;
        return fail(nullptr, HLBM_ENOMEM, "host allocation failed");
    }
    set_phase(c, 0);
    *out = c;
    return HLBM_OK;
}

int hlbm_step(hlbm_ctx *c, int n_coarse)
{
    if (!c) return HLBM_EINVAL;
    if (c->timing_dirty) return fail(c, HLBM_ESTATE, "the state was consumed by hlbm_time_kernel");
    if (n_coarse < 0) return fail(c, HLBM_EINVAL, "n_coarse must be >= 0");
    Range r("hlbm_step");
    try {
        for (int k = 0; k < n_coarse; k++) {
            if (c->use_graphs) {
                // two steps per launch where they remain and no health check falls between them
                const bool pair = c->graph2[c->steps & 1] && k + 1 < n_coarse &&
                                  !(c->check_every > 0 && (c->steps + 1) % c->check_every == 0);
                if (pair) {
                    ck(cudaGraphLaunch(c->graph2[c->steps & 1], c->stream), "graph launch");
                    c->steps++;
                    k++;
                } else {
                    ck(cudaGraphLaunch(c->graph[c->steps & 1], c->stream), "graph launch");
                }
            } else {
                set_phase(c, c->steps);
                enqueue_coarse_step(c, c->stream);
                ck(cudaGetLastError(), "kernel launch");
            }
            c->steps++;
            set_phase(c, c->steps);
            if (c->check_every > 0 && (c->steps % c->check_every) == 0) {
                int flag = 0;
                ck(cudaMemcpyAsync(&flag, c->dev.flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flag");
                ck(cudaStreamSynchronize(c->stream), "sync");
                if (flag & 2) return fail(c, HLBM_ETIMEOUT, "a device-side wait gave up (operator copy did not arrive)");
                if (flag) return fail(c, HLBM_EUNSTABLE, "NaN in the force reduction: the simulation is unstable");
                const double m = level0_mass(c);
                c->mass_drift = std::fabs(m - c->mass0) / c->mass0;
                if (!(c->mass_drift <= kMassDriftLimit))
                    return fail(c, HLBM_EUNSTABLE, "total mass drifted by " + std::to_string(c->mass_drift) +
                                                       " of the initial mass: the simulation is unstable");
            }
        }
    } catch (const CudaError &e) {
        return fail(c, HLBM_ECUDA, e.msg);
    }
    return HLBM_OK;
}

int hlbm_forces(hlbm_ctx *c, double *cd, double *cl, int cap, int *n_written)
{
    if (!c || !n_written || (cap > 0 && (!cd || !cl))) return c ? fail(c, HLBM_EINVAL, "bad arguments") : HLBM_EINVAL;
    *n_written = 0;
    if (c->dev.m.n == 0) return HLBM_OK;
    try {
        int counter = 0;
        ck(cudaMemcpyAsync(&counter, c->dev.force_counter, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "counter");
        ck(cudaStreamSynchronize(c->stream), "sync");
        long first = std::max<long>(c->forces_read, long(counter) - c->dev.force_cap);
        long n = std::min<long>(long(counter) - first, cap);
        if (n <= 0) return HLBM_OK;
        // only the n samples read: slots first .. first + n - 1 of the ring,
        // at most two contiguous runs
        std::vector<double> buf(size_t(2) * n);
        const long s0 = first % c->dev.force_cap, n0 = std::min<long>(n, c->dev.force_cap - s0);
        ck(cudaMemcpyAsync(buf.data(), c->dev.force_buf + 2 * s0, size_t(2) * n0 * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream), "forces");
        if (n > n0)
            ck(cudaMemcpyAsync(buf.data() + 2 * n0, c->dev.force_buf, size_t(2) * (n - n0) * sizeof(double),
                               cudaMemcpyDeviceToHost, c->stream), "forces");
        ck(cudaStreamSynchronize(c->stream), "sync");
        for (long k = 0; k < n; k++) {
            cd[k] = buf[2 * k];
            cl[k] = buf[2 * k + 1];
        }
        c->forces_read = first + n;
        *n_written = int(n);
    } catch (const CudaError &e) {
        return fail(c, HLBM_ECUDA, e.msg);
    }
    return HLBM_OK;
}

static void fields_dispatch(hlbm_ctx *c, int grid, double *rho, double *ux, double *uy, double *pop)
{
    if (c->plan.precision == HLBM_FP32) launch_fields<float, float>(c->dev, grid, rho, ux, uy, pop, c->stream);
    else if (c->plan.precision == HLBM_FP16S) launch_fields<float, __half>(c->dev, grid, rho, ux, uy, pop, c->stream);
    else launch_fields<double, double>(c->dev, grid, rho, ux, uy, pop, c->stream);
}

static int readback(hlbm_ctx *c, int grid, double *rho, double *ux, double *uy, double *pop, size_t cap)
{
    if (!c) return HLBM_EINVAL;
    size_t n;
    if (grid == -1) n = size_t(c->plan.n);
    else if (grid >= 0 && grid < c->plan.L) n = size_t(c->plan.lv[grid].nx) * c->plan.lv[grid].ny;
    else return fail(c, HLBM_EINVAL, "grid out of range");
    size_t need = pop ? 9 * n : n;
    if (cap < need) return fail(c, HLBM_EINVAL, "output capacity too small");
    if (n == 0) return HLBM_OK;
    try {
        double *d = c->d_out;
        if (pop) {
            fields_dispatch(c, grid, nullptr, nullptr, nullptr, d);
            ck(cudaGetLastError(), "fields kernel");
            ck(cudaMemcpyAsync(pop, d, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "D2H");
        } else {
            fields_dispatch(c, grid, d, d + n, d + 2 * n, nullptr);
            ck(cudaGetLastError(), "fields kernel");
            if (rho) ck(cudaMemcpyAsync(rho, d, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "D2H");
            if (ux) ck(cudaMemcpyAsync(ux, d + n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "D2H");
            if (uy) ck(cudaMemcpyAsync(uy, d + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "D2H");
        }
        ck(cudaStreamSynchronize(c->stream), "sync");
    } catch (const CudaError &e) {
        return fail(c, HLBM_ECUDA, e.msg);
    }
    return HLBM_OK;
}

int hlbm_fields(hlbm_ctx *c, int grid, double *rho, double *ux, double *uy, size_t cap)
{
    return readback(c, grid, rho, ux, uy, nullptr, cap);
}

int hlbm_populations(hlbm_ctx *c, int grid, double *out, size_t cap)
{
    if (!out) return c ? fail(c, HLBM_EINVAL, "out is NULL") : HLBM_EINVAL;
    return readback(c, grid, nullptr, nullptr, nullptr, out, cap);
}

int hlbm_info(const hlbm_ctx *c, const char *key, double *value)
{
    if (!c || !key || !value) return HLBM_EINVAL;
    const Plan &P = c->plan;
    std::string k(key);
    if (k == "n_sub") *value = P.n_sub;
    else if (k == "n_levels") *value = P.L;
    else if (k == "tau_u") *value = P.tau_u;
    else if (k.size() == 4 && k.compare(0, 3, "tau") == 0 && k[3] >= '0' && k[3] < '0' + P.L) *value = P.lv[k[3] - '0'].tau;
    else if (k == "steps") *value = double(c->steps);
    else if (k == "n_interp") *value = double(P.is_node.size());
    else if (k == "n_ring") *value = P.n_ring;
    else if (k == "n_wall_edges") *value = double(P.wea.size());
    else if (k == "nnz") *value = double(P.col.size());
    else if (k == "lattice_updates") {
        double u = 0;
        for (int l = 0; l < P.L; l++) {
            double nn = double(P.lv[l].nx) * P.lv[l].ny;
            for (size_t y = 0; y < P.lv[l].hx0.size(); y++) nn -= P.lv[l].hx1[y] - P.lv[l].hx0[y];
            u += nn * double(1L << l);
        }
        *value = u;
    } else if (k == "fv_updates") *value = double(P.n) * P.n_sub * double(1L << (P.L - 1));
    else if (k == "launches_per_step") *value = double(c->launches_per_step);
    else if (k == "fv_tiles") *value = double(c->dev.m.tl.n_tiles);
    else if (k == "mass" || k == "mass_drift") {
        if (c->timing_dirty) return HLBM_ESTATE;
        try {
            const double m = level0_mass(const_cast<hlbm_ctx *>(c));
            *value = k == "mass" ? m : std::fabs(m - c->mass0) / c->mass0;
        } catch (const CudaError &) {
            return HLBM_ECUDA;
        }
    }
    else if (k == "bounds_violations" || k == "bounds_sites") {
        unsigned int b[2];
        if (cudaDeviceSynchronize() != cudaSuccess) return HLBM_ECUDA;
        *value = debug_bounds(b) ? double(b[k == "bounds_sites"]) : -1.0;
    }
    else if (k == "fv_variant")
        *value = double(c->dev.m.fv_variant + (c->dev.m.tl.rows == kTileRowsWide ? 4 : 0));
    else if (k == "fv_tile_rows") *value = double(c->dev.m.tl.rows);
    else if (k == "fv_filter") *value = c->dev.fv_filter;
    else if (k == "create_ms_setup") *value = c->create_ms[0];
    else if (k == "create_ms_device") *value = c->create_ms[1];
    else if (k == "create_ms_capture") *value = c->create_ms[2];
    else if (k == "create_ms_upload") *value = c->build_ms[0];
    else if (k == "create_ms_init") *value = c->build_ms[1];
    else if (k == "fv_tune_us1") *value = c->fv_tune_us[0];
    else if (k == "fv_tune_us2") *value = c->fv_tune_us[1];
    else if (k == "fv_tune_us3") *value = c->fv_tune_us[2];
    else if (k == "fv_tune_us4") *value = c->fv_tune_us[3];
    else if (k == "fv_tune_us5") *value = c->fv_tune_us[4];
    else if (k == "fv_tune_us6") *value = c->fv_tune_us[5];
    else if (k == "fv_tune_us7") *value = c->fv_tune_us[6];
    else if (k == "fv_tune_us8") *value = c->fv_tune_us[7];
    else if (k == "fv_smem") *value = double(c->dev.m.tl.smem_bytes);
    else if (k == "fv_bytes") {
        // algorithmic bytes of one finite-volume sub-step: the 9 state values of
        // every node read and written, one (s_x, s_y, C, column) entry per
        // off-diagonal operator coefficient
        double vb = P.precision == HLBM_FP64 ? 8.0 : 4.0;  // the mesh is FP32 in FP16S mode
        *value = double(P.n) * 18.0 * vb + double(P.col.size() - size_t(P.n)) * 4.0 * vb;
    } else if (k.size() == 14 && k.compare(0, 13, "collide_bytes") == 0) {
        int l = k[13] - '0';
        if (l < 0 || l >= P.L) return HLBM_EINVAL;
        double nn = double(P.lv[l].nx) * P.lv[l].ny;
        for (size_t y = 0; y < P.lv[l].hx0.size(); y++) nn -= P.lv[l].hx1[y] - P.lv[l].hx0[y];
        *value = nn * 18.0 * (P.precision == HLBM_FP64 ? 8.0 : (P.precision == HLBM_FP32 ? 4.0 : 2.0));
    }
    else return HLBM_EINVAL;
    return HLBM_OK;
}

int hlbm_inspect(const hlbm_level *lv, int n_levels, const hlbm_mesh *m, double Re, double Ma, double aoa_deg,
                 const hlbm_options *opt, const char *table, double *out, size_t cap, size_t *n)
{
    if (!table || !n) return fail(nullptr, HLBM_EINVAL, "table and n are required");
    Plan P;
    std::string err;
    int rc;
    try {
        rc = build_plan(lv, n_levels, m, Re, Ma, aoa_deg, opt, P, err);
    } catch (const std::bad_alloc &) {
        return fail(nullptr, HLBM_ENOMEM, "host allocation failed");
    }
    if (rc != HLBM_OK) return fail(nullptr, rc, err);
    std::vector<double> v;
    std::string t(table);
    auto put_i = [&](const std::vector<int> &a) { v.assign(a.begin(), a.end()); };
    if (t == "rowptr") put_i(P.rowptr);
    else if (t == "col") put_i(P.col);
    else if (t == "perm") put_i(P.perm);
    else if (t == "wall_geo") v = P.wall_geo;
    else if (t == "perm") put_i(P.perm);
    else if (t == "wall_geo") v = P.wall_geo;
    else if (t == "sx") v = P.sx;
    else if (t == "sy") v = P.sy;
    else if (t == "cc") v = P.cc;
    else if (t == "area") v = P.area;
    else if (t == "xy") v = P.xy;
    else if (t == "is_node") put_i(P.is_node);
    else if (t == "is_don") put_i(P.is_don);
    else if (t == "is_w") v = P.is_w;
    else if (t == "ring") put_i(P.ring);
    else if (t == "ring_don") put_i(P.ring_don);
    else if (t == "ring_w") v = P.ring_w;
    else if (t == "wall_edges") {
        for (size_t e = 0; e < P.wea.size(); e++) { v.push_back(P.wea[e]); v.push_back(P.web[e]); }
    } else if (t == "n_sub") v.assign(1, double(P.n_sub));
    else if (t.size() == 9 && t.compare(0, 8, "inactive") == 0 && t[8] >= '0' && t[8] < '0' + P.L) {
        const LevelPlan &l = P.lv[t[8] - '0'];
        v.assign(size_t(l.nx) * l.ny, 0.0);
        for (size_t y = 0; y < l.hx0.size(); y++)
            for (int x = l.hx0[y]; x < l.hx1[y]; x++) v[y * l.nx + x] = 1.0;
    }
    else return fail(nullptr, HLBM_EINVAL, "unknown table");
    *n = v.size();
    if (out) {
        if (cap < v.size()) return fail(nullptr, HLBM_EINVAL, "output capacity too small");
        std::copy(v.begin(), v.end(), out);
    }
    return HLBM_OK;
}

int hlbm_time_kernel(hlbm_ctx *c, const char *kernel, int reps, double *avg_ms)
{
    if (!c || !kernel || !avg_ms || reps < 1) return c ? fail(c, HLBM_EINVAL, "bad arguments") : HLBM_EINVAL;
    std::string k(kernel);
    int lvl = -1;
    if (k == "fv") {
        if (c->dev.m.n == 0) return fail(c, HLBM_EINVAL, "no mesh");
    } else if (k.size() == 8 && k.compare(0, 7, "collide") == 0 && k[7] >= '0' && k[7] < '0' + c->plan.L) {
        lvl = k[7] - '0';
    } else {
        return fail(c, HLBM_EINVAL, "unknown kernel");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    try {
        ck(cudaEventCreate(&e0), "event");
        ck(cudaEventCreate(&e1), "event");
        const int prec = c->plan.precision;
        auto one = [&](int r) {
            if (lvl < 0) {
                int m = r % std::max(1, c->dev.n_sub);
                if (prec == HLBM_FP64) launch_fv<double, double>(c->dev, m, c->stream);
                else launch_fv<float, float>(c->dev, m, c->stream);
                c->dev.m.gcur ^= 1;
            } else {
                if (prec == HLBM_FP32) launch_collide<float, float>(c->dev, lvl, c->stream);
                else if (prec == HLBM_FP16S) launch_collide<float, __half>(c->dev, lvl, c->stream);
                else launch_collide<double, double>(c->dev, lvl, c->stream);
                c->dev.lv[lvl].parity ^= 1;
            }
        };
        // the repetitions are captured as one CUDA graph so that the GPU runs
        // them back to back (timing individual launches from the host would
        // measure the launch rate once a kernel is faster than it)
        ck(cudaStreamSynchronize(c->stream), "sync");
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        ck(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaStream_t user = c->stream;
        c->stream = c->cap_stream;
        for (int r = 0; r < reps; r++) one(r);
        c->stream = user;
        ck(cudaStreamEndCapture(c->cap_stream, &graph), "end capture");
        ck(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate");
        cudaGraphDestroy(graph);
        ck(cudaGraphLaunch(exec, c->stream), "graph launch");  // warm-up
        ck(cudaEventRecord(e0, c->stream), "record");
        ck(cudaGraphLaunch(exec, c->stream), "graph launch");
        ck(cudaEventRecord(e1, c->stream), "record");
        ck(cudaEventSynchronize(e1), "sync");
        cudaGraphExecDestroy(exec);
        float ms = 0;
        ck(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
        *avg_ms = double(ms) / reps;
        ck(cudaGetLastError(), "kernel launch");
    } catch (const CudaError &e) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return fail(c, HLBM_ECUDA, e.msg);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->timing_dirty = true;
    return HLBM_OK;
}

int hlbm_sync(hlbm_ctx *c)
{
    if (!c) return HLBM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, HLBM_ECUDA, cudaGetErrorString(e));
    return HLBM_OK;
}

int hlbm_destroy(hlbm_ctx *c)
{
    if (!c) return HLBM_OK;
    if (c->shadow) {
        release(c->shadow);
        delete c->shadow;
        c->shadow = nullptr;
    }
    release(c);
    delete c;
    return HLBM_OK;
}

int hlbm_wall_stats(hlbm_ctx *c, double *out, size_t cap, int *n_wall, long *n_samples)
{
    if (!c || !n_wall || !n_samples) return c ? fail(c, HLBM_EINVAL, "n_wall and n_samples are required") : HLBM_EINVAL;
    const DevMesh &M = c->dev.m;
    if (!M.wall_stats) return fail(c, HLBM_ESTATE, "the context was created without wall_stats");
    const int nw = c->plan.n_wall;
    *n_wall = nw;
    *n_samples = c->steps - c->stats_base;
    if (!out) return HLBM_OK;
    if (cap < 10 * size_t(nw)) return fail(c, HLBM_EINVAL, "output capacity too small");
    if (c->timing_dirty) return fail(c, HLBM_ESTATE, "the state was consumed by hlbm_time_kernel");
    std::vector<double> acc(3 * size_t(nw));
    try {
        if (nw > 0) {
            ck(cudaMemcpyAsync(acc.data(), M.wall_acc, acc.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
               "D2H");
            ck(cudaStreamSynchronize(c->stream), "sync");
        }
    } catch (const CudaError &e) {
        return fail(c, HLBM_ECUDA, e.msg);
    }
    const double inv = *n_samples > 0 ? 1.0 / double(*n_samples) : 0.0;
    for (int w = 0; w < nw; w++) {
        const double *g = &c->plan.wall_geo[7 * size_t(w)];
        double *r = out + 10 * size_t(w);
        r[0] = g[0];
        r[1] = g[1];
        r[2] = acc[w] * inv;
        r[3] = acc[size_t(nw) + w] * inv;
        r[4] = acc[2 * size_t(nw) + w] * inv;
        for (int k = 0; k < 5; k++) r[5 + k] = g[2 + k];
    }
    return HLBM_OK;
}

}  // extern "C"

namespace {

// Device tables of the finite-volume adjoint, from the plan (device order).
void build_adjoint_tables(hlbm_ctx *c)
{
    const Plan &P = c->plan;
    AdjTables &A = c->adj;
    const double dt = 1.0 / P.n_sub, dt_tau = dt / P.tau_u;
    std::vector<int> rp(size_t(P.n) + 1, 0), rcol, rcsr;
    std::vector<double> rcoef;
    for (int r = 0; r < P.n; r++) {
        const int old = P.perm[r];
        for (int k = P.rowptr[old]; k < P.rowptr[old + 1]; k++) {
            if (P.col[k] == old) continue;
            rcol.push_back(P.inv[P.col[k]]);
            rcsr.push_back(k);
            rcoef.push_back(dt * P.sx[k]);
            rcoef.push_back(dt * P.sy[k]);
            rcoef.push_back(dt_tau * P.cc[k]);
        }
        rp[r + 1] = int(rcol.size());
    }
    // transposed: for each node, the rows that read it (its own first)
    std::vector<int> tp(size_t(P.n) + 1, 0), trow, tpos;
    for (int r = 0; r < P.n; r++) {
        tp[r + 1]++;
        for (int e = rp[r]; e < rp[r + 1]; e++) tp[rcol[e] + 1]++;
    }
    for (int r = 0; r < P.n; r++) tp[r + 1] += tp[r];
    trow.resize(tp[P.n]);
    tpos.resize(tp[P.n]);
    std::vector<int> fill(tp.begin(), tp.end() - 1);
    for (int r = 0; r < P.n; r++) {
        trow[fill[r]] = r;
        tpos[fill[r]++] = -1;
    }
    for (int r = 0; r < P.n; r++)
        for (int e = rp[r]; e < rp[r + 1]; e++) {
            const int q = rcol[e];
            trow[fill[q]] = r;
            tpos[fill[q]++] = e - rp[r];
        }
    // wall edges in device order and the edges of each node
    const int ne = int(P.wea.size());
    std::vector<int> wea(ne), web(ne), wptr(size_t(P.n) + 1, 0), wedge;
    std::vector<double> wn(2 * size_t(ne));
    for (int e = 0; e < ne; e++) {
        wea[e] = P.inv[P.wea[e]];
        web[e] = P.inv[P.web[e]];
        wn[2 * e] = -(P.xy[2 * P.web[e] + 1] - P.xy[2 * P.wea[e] + 1]);  // left normal: into the fluid
        wn[2 * e + 1] = P.xy[2 * P.web[e]] - P.xy[2 * P.wea[e]];
        wptr[wea[e] + 1]++;
        wptr[web[e] + 1]++;
    }
    for (int r = 0; r < P.n; r++) wptr[r + 1] += wptr[r];
    wedge.resize(wptr[P.n]);
    std::vector<int> wf(wptr.begin(), wptr.end() - 1);
    for (int e = 0; e < ne; e++) {
        wedge[wf[wea[e]]++] = e;
        wedge[wf[web[e]]++] = e;
    }
    A.rp = upload(c, rp);
    A.rcol = upload(c, rcol);
    A.rcsr = upload(c, rcsr);
    A.rcoef = upload(c, rcoef);
    A.tp = upload(c, tp);
    A.trow = upload(c, trow);
    A.tpos = upload(c, tpos);
    A.n_edges = ne;
    A.wea = upload(c, wea);
    A.web = upload(c, web);
    A.wn = upload(c, wn);
    A.wptr = upload(c, wptr);
    A.wedge = upload(c, wedge);
    A.perm = upload(c, P.perm);
    // geometry tables, input node order
    std::vector<double> pcoef(3 * P.col.size());
    for (size_t e = 0; e < P.col.size(); e++) {
        pcoef[3 * e] = P.sx[e];
        pcoef[3 * e + 1] = P.sy[e];
        pcoef[3 * e + 2] = P.cc[e];
    }
    std::vector<int> ntp(size_t(P.n) + 1, 0), ntl(3 * size_t(P.ntri));
    for (int k = 0; k < 3 * P.ntri; k++) ntp[P.tri[k] + 1]++;
    for (int r = 0; r < P.n; r++) ntp[r + 1] += ntp[r];
    {
        std::vector<int> f(ntp.begin(), ntp.end() - 1);
        for (int k = 0; k < 3 * P.ntri; k++) ntl[f[P.tri[k]]++] = k / 3;
    }
    // boundary edges: directed triangle edges a -> b whose reverse is absent
    std::vector<uint64_t> keys(3 * size_t(P.ntri));
    auto key = [](int a, int b) { return (uint64_t(uint32_t(a)) << 32) | uint32_t(b); };
    for (int t = 0; t < P.ntri; t++)
        for (int a = 0; a < 3; a++) keys[3 * size_t(t) + a] = key(P.tri[3 * t + a], P.tri[3 * t + (a + 1) % 3]);
    std::vector<uint64_t> sorted(keys);
    std::sort(sorted.begin(), sorted.end());
    std::vector<int> bed, bptr(size_t(P.n) + 1, 0), blist;
    for (int t = 0; t < P.ntri; t++)
        for (int a = 0; a < 3; a++) {
            const int ia = P.tri[3 * t + a], ib = P.tri[3 * t + (a + 1) % 3];
            if (std::binary_search(sorted.begin(), sorted.end(), key(ib, ia))) continue;
            bed.push_back(ia);
            bed.push_back(ib);
        }
    const int nb = int(bed.size() / 2);
    for (int b = 0; b < nb; b++) {
        bptr[bed[2 * b] + 1]++;
        bptr[bed[2 * b + 1] + 1]++;
    }
    for (int r = 0; r < P.n; r++) bptr[r + 1] += bptr[r];
    blist.resize(bptr[P.n]);
    {
        std::vector<int> f(bptr.begin(), bptr.end() - 1);
        for (int b = 0; b < nb; b++) {
            blist[f[bed[2 * b]]++] = b;
            blist[f[bed[2 * b + 1]]++] = b;
        }
    }
    std::vector<int> iwptr(size_t(P.n) + 1, 0), iwlist;
    for (int e = 0; e < ne; e++) {
        iwptr[P.wea[e] + 1]++;
        iwptr[P.web[e] + 1]++;
    }
    for (int r = 0; r < P.n; r++) iwptr[r + 1] += iwptr[r];
    iwlist.resize(iwptr[P.n]);
    {
        std::vector<int> f(iwptr.begin(), iwptr.end() - 1);
        for (int e = 0; e < ne; e++) {
            iwlist[f[P.wea[e]]++] = e;
            iwlist[f[P.web[e]]++] = e;
        }
    }
    A.n_tri = P.ntri;
    A.n_bedge = nb;
    A.prow = upload(c, P.rowptr);
    A.pcol = upload(c, P.col);
    A.pcoef = upload(c, pcoef);
    A.parea = upload(c, P.area);
    A.pxy = upload(c, P.xy);
    A.ptri = upload(c, P.tri);
    A.ntp = upload(c, ntp);
    A.ntl = upload(c, ntl);
    A.bed = upload(c, bed);
    A.bptr = upload(c, bptr);
    A.blist = upload(c, blist);
    A.iwea = upload(c, P.wea);
    A.iweb = upload(c, P.web);
    A.iwptr = upload(c, iwptr);
    A.iwlist = upload(c, iwlist);
    A.inv = upload(c, P.inv);
    A.built = true;
}

// Tables of the coupled-step adjoint (single level): Eq. 9 and Eq. 8 donor
// pairs transposed to the donors.
void build_coupled_tables(hlbm_ctx *c)
{
    const Plan &P = c->plan;
    AdjTables &A = c->adj;
    const LevelPlan &F = P.lv[P.L - 1];
    const size_t nl = size_t(F.nx) * F.ny;
    std::vector<int> lptr(nl + 1, 0), lent(P.ring_don.size());
    for (int d : P.ring_don) lptr[size_t(d) + 1]++;
    for (size_t k = 0; k < nl; k++) lptr[k + 1] += lptr[k];
    {
        std::vector<int> f(lptr.begin(), lptr.end() - 1);
        for (size_t t = 0; t < P.ring_don.size(); t++) lent[f[P.ring_don[t]]++] = int(t);
    }
    std::vector<int> hptr(size_t(P.n) + 1, 0), hent(P.is_don.size());
    for (int d : P.is_don) hptr[P.inv[d] + 1]++;
    for (int k = 0; k < P.n; k++) hptr[k + 1] += hptr[k];
    {
        std::vector<int> f(hptr.begin(), hptr.end() - 1);
        for (size_t t = 0; t < P.is_don.size(); t++) hent[f[P.inv[P.is_don[t]]]++] = int(t);
    }
    A.lptr = upload(c, lptr);
    A.lent = upload(c, lent);
    A.hptr = upload(c, hptr);
    A.hent = upload(c, hent);
    {
        std::vector<double> isxy(2 * P.is_node.size());
        for (size_t k = 0; k < P.is_node.size(); k++) {
            isxy[2 * k] = double(P.is_node[k] % F.nx);
            isxy[2 * k + 1] = double(P.is_node[k] / F.nx);
        }
        A.isd_in = upload(c, P.is_don);
        A.is_xy = upload(c, isxy);
    }
    // prolongation into level l: each fine perimeter node reads 1 (even
    // position) or 3 (odd: weights -1/8, 3/4, 3/8) band entries of level l - 1
    for (int l = 1; l < P.L; l++) {
        const LevelPlan &fl = P.lv[l], &pl = P.lv[l - 1];
        const int nx = fl.nx, ny = fl.ny, w = pl.cmx + 2, h = pl.cmy + 2, band_n = 2 * w + 2 * h;
        const int nper = 2 * nx + 2 * (ny - 2);
        std::vector<std::vector<std::pair<int, double>>> by(band_n);
        for (int k = 0; k < nper; k++) {
            int i, j;
            if (k < nx) { i = k; j = 0; }
            else if (k < 2 * nx) { i = k - nx; j = ny - 1; }
            else if (k < 2 * nx + ny - 2) { i = 0; j = k - 2 * nx + 1; }
            else { i = nx - 1; j = k - 2 * nx - (ny - 2) + 1; }
            int base, pos, odd;
            if (j == 0 || j == ny - 1) { base = (j == 0) ? 0 : w; pos = (i >> 1) + 1; odd = i & 1; }
            else { base = 2 * w + ((i == 0) ? 0 : h); pos = (j >> 1) + 1; odd = j & 1; }
            for (int t = 0; t < (odd ? 3 : 1); t++) {
                const int b = base + pos + (odd ? t - 1 : 0);
                const double wk = odd ? (t == 0 ? -0.125 : (t == 1 ? 0.75 : 0.375)) : 1.0;
                if (b < 0 || b >= band_n) throw CudaError{"prolongation band index out of range"};
                by[b].push_back({k, wk});
            }
        }
        std::vector<int> pp(size_t(band_n) + 1, 0), pk;
        std::vector<double> pw;
        for (int b = 0; b < band_n; b++) {
            for (auto &e : by[b]) {
                pk.push_back(e.first);
                pw.push_back(e.second);
            }
            pp[b + 1] = int(pk.size());
        }
        A.pp[l] = upload(c, pp);
        A.pk[l] = upload(c, pk);
        A.pw[l] = upload(c, pw);
    }
    A.coupled_built = true;
}

}  // namespace

extern "C" {

int hlbm_fv_adjoint(hlbm_ctx *c, int n_window, double wd, double wl, double *J, double *grad_g, size_t cap_g,
                    double *grad_coef, size_t cap_coef, double *grad_xy, size_t cap_xy, double *dJ_daoa)
{
    if (!c) return HLBM_EINVAL;
    const Plan &P = c->plan;
    if (P.precision != HLBM_FP64) return fail(c, HLBM_ENOTIMPL, "the finite-volume adjoint runs on FP64 contexts");
    if (c->dev.fv_filter > 0.0) return fail(c, HLBM_ENOTIMPL, "the adjoint does not cover the fv_filter option");
    if (P.n == 0) return fail(c, HLBM_EINVAL, "the context has no mesh");
    if (n_window < 1 || n_window > P.n_sub) return fail(c, HLBM_EINVAL, "n_window must be in 1..n_sub");
    if (!J) return fail(c, HLBM_EINVAL, "J is NULL");
    if (grad_g && cap_g < 9 * size_t(P.n)) return fail(c, HLBM_EINVAL, "grad_g capacity below 9 n");
    if (grad_coef && cap_coef < 3 * P.col.size()) return fail(c, HLBM_EINVAL, "grad_coef capacity below 3 nnz");
    if (grad_xy && cap_xy < 2 * size_t(P.n)) return fail(c, HLBM_EINVAL, "grad_xy capacity below 2 n");
    if (c->timing_dirty) return fail(c, HLBM_ESTATE, "the state was consumed by hlbm_time_kernel");
    Range r("hlbm_fv_adjoint");
    DevCtx &D = c->dev;
    const int Np = D.m.Np, n = P.n, M = n_window;
    const size_t plane = size_t(9) * Np;
    std::vector<void *> scratch;
    auto scr = [&](size_t bytes) {
        void *p = dalloc(c, bytes);
        scratch.push_back(p);
        return p;
    };
    int rc = HLBM_OK;
    try {
        if (!c->adj.built) build_adjoint_tables(c);
        const AdjTables &A = c->adj;
        double *st = (double *)scr((size_t(M) + 1) * plane * sizeof(double));  // states g_0 .. g_M
        double *lam = (double *)scr(2 * plane * sizeof(double));
        double *rs = (double *)scr(3 * plane * sizeof(double));  // reverse sub-step scratch
        double *gc = (double *)scr(std::max<size_t>(1, 3 * P.col.size()) * sizeof(double));
        double *gg = (double *)scr(9 * size_t(n) * sizeof(double));
        double *dJ = (double *)scr(2 * sizeof(double));  // J, dJ/d(angle of attack)
        const bool geo = grad_xy || dJ_daoa;
        double *gxy = geo ? (double *)scr(2 * size_t(n) * sizeof(double)) : nullptr;
        double *gs = geo ? (double *)scr((3 * size_t(n) + 2 * size_t(std::max(1, c->adj.n_edges))) * sizeof(double))
                         : nullptr;
        cudaStream_t s = c->stream;
        ck(cudaMemsetAsync(st, 0, (size_t(M) + 1) * plane * sizeof(double), s), "memset");
        ck(cudaMemsetAsync(gc, 0, 3 * P.col.size() * sizeof(double), s), "memset");
        ck(cudaMemcpyAsync(st, D.m.g[D.m.gcur], plane * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
        // forward window with the production sub-step kernel; the interface
        // rows take the current Eq. 9 data (Q0) at every sub-step
        DevCtx W = D;
        W.m.Q1 = W.m.Q0;
        W.m.gcur = 0;
        for (int m = 0; m < M; m++) {
            W.m.g[0] = st + size_t(m) * plane;
            W.m.g[1] = st + size_t(m + 1) * plane;
            launch_fv<double, double>(W, m, s);
        }
        ck(cudaGetLastError(), "forward window");
        const double inv_q = 1.0 / P.qdyn;
        const double *gM = st + size_t(M) * plane;
        launch_adj_value(A, gM, Np, wd, wl, inv_q, dJ, s);
        launch_adj_terminal(A, gM, Np, n, wd, wl, inv_q, lam, s);
        const double dt = 1.0 / P.n_sub, dt_tau = dt / P.tau_u, csP = dt_tau * (11.0 / 18.0);
        for (int m = M - 1; m >= 0; m--) {
            const double *lin = lam + size_t((M - 1 - m) & 1) * plane;
            double *lout = lam + size_t((M - m) & 1) * plane;
            launch_fv_adjoint(A, st + size_t(m) * plane, Np, n, csP, P.n_wall, P.ring_start,
                              m < P.n_sub - 1 ? 1 : 0, dt, dt_tau, lin, lout, gc, rs, s);
        }
        const double *lam0 = lam + size_t(M & 1) * plane;
        launch_adj_populations(A, st, Np, n, lam0, gg, s);
        if (geo) {
            const double al = P.aoa_deg * M_PI / 180.0;
            launch_adj_geometry(A, n, gc, gM, Np, wd, wl, inv_q, std::cos(al), std::sin(al), P.pivot[0], P.pivot[1],
                                gs, gxy, dJ + 1, s);
        }
        ck(cudaGetLastError(), "adjoint kernels");
        ck(cudaMemcpyAsync(J, dJ, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
        if (grad_g) ck(cudaMemcpyAsync(grad_g, gg, 9 * size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
        if (grad_coef)
            ck(cudaMemcpyAsync(grad_coef, gc, 3 * P.col.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
        if (grad_xy) ck(cudaMemcpyAsync(grad_xy, gxy, 2 * size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
        if (dJ_daoa) ck(cudaMemcpyAsync(dJ_daoa, dJ + 1, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
        ck(cudaStreamSynchronize(s), "sync");
        int flag = 0;
        ck(cudaMemcpy(&flag, D.flag, sizeof(int), cudaMemcpyDeviceToHost), "flag");
        if (flag & 2) rc = fail(c, HLBM_ETIMEOUT, "a device-side wait gave up (operator copy did not arrive)");
    } catch (const CudaError &e) {
        rc = fail(c, HLBM_ECUDA, e.msg);
    } catch (const std::bad_alloc &) {
        rc = fail(c, HLBM_ENOMEM, "host allocation failed");
    }
    for (void *p : scratch) dfree(c, p);
    return rc;
}

namespace {
// The FP64 twin of an FP32 context: the same plan built with FP64 device
// tables (Eq. 3 entries, Eq. 8 and Eq. 9 weights, ...) and its own FP64
// adjoint tables, for the reverse sweep of an adjoint whose forward steps run
// in FP32.  Shares the caller's stream and allocator; freed with the context.
void make_shadow(hlbm_ctx *c)
{
    hlbm_ctx *t = new hlbm_ctx();
    t->plan = c->plan;
    t->plan.precision = HLBM_FP64;
    t->stream = c->stream;
    t->alloc_fn = c->alloc_fn;
    t->free_fn = c->free_fn;
    t->alloc_ctx = c->alloc_ctx;
    t->dev.force_cap = 1;
    try {
        build_device<double, double>(t);
    } catch (...) {
        release(t);
        delete t;
        throw;
    }
    c->shadow = t;
}
}  // namespace

int hlbm_adjoint(hlbm_ctx *c, int n_steps, int n_skip, double wd, double wl, double *J, double *grad_lattice,
                 size_t cap_lat, double *grad_mesh, size_t cap_mesh, double *grad_xy, size_t cap_xy, double *dJ_daoa)
{
    if (!c) return HLBM_EINVAL;
    const Plan &P = c->plan;
    if (P.precision == HLBM_FP16S) return fail(c, HLBM_ENOTIMPL, "the adjoint runs on FP64 and FP32 contexts");
    if (c->dev.fv_filter > 0.0) return fail(c, HLBM_ENOTIMPL, "the adjoint does not cover the fv_filter option");
    if (P.n == 0) return fail(c, HLBM_EINVAL, "the context has no mesh");
    if (n_steps < 1) return fail(c, HLBM_EINVAL, "n_steps must be >= 1");
    if (n_skip < 0 || n_skip >= n_steps) return fail(c, HLBM_EINVAL, "n_skip must be in 0..n_steps-1");
    if (!J) return fail(c, HLBM_EINVAL, "J is NULL");
    size_t lat_total = 0;  // populations of all levels
    for (int l = 0; l < P.L; l++) lat_total += 9 * size_t(P.lv[l].nx) * P.lv[l].ny;
    if (grad_lattice && cap_lat < lat_total) return fail(c, HLBM_EINVAL, "grad_lattice capacity below 9 sum nx ny");
    if (grad_mesh && cap_mesh < 9 * size_t(P.n)) return fail(c, HLBM_EINVAL, "grad_mesh capacity below 9 n");
    if (grad_xy && cap_xy < 2 * size_t(P.n)) return fail(c, HLBM_EINVAL, "grad_xy capacity below 2 n");
    if (c->timing_dirty) return fail(c, HLBM_ESTATE, "the state was consumed by hlbm_time_kernel");
    Range r("hlbm_adjoint");
    const bool geo = grad_xy || dJ_daoa;
    const int K = n_steps, n = P.n, ns = P.n_sub, L = P.L;
    const double wavg = 1.0 / (K - n_skip);  // weight of each averaged force sample
    const long k0 = c->steps;
    std::vector<void *> scratch;
    auto scr = [&](size_t bytes) {
        void *p = dalloc(c, bytes);
        scratch.push_back(p);
        return (double *)p;
    };
    int rc = HLBM_OK;
    const DevCtx D0 = c->dev;
    const long launches0 = c->launches, lps0 = c->launches_per_step;
    bool side0[hlbm::kMaxLevels];
    std::copy(c->side_ok, c->side_ok + hlbm::kMaxLevels, side0);
    // FP32 contexts: the forward steps (checkpointed passes and recorded
    // steps) run in FP32 on the context's own kernels; every recorded buffer
    // is widened to FP64, and the reverse sweep (the finite-volume groups it
    // recomputes, every adjoint kernel and all gradient sums) runs in FP64
    // with the tables of an FP64 twin of the context
    const bool f32 = P.precision == HLBM_FP32;
    const size_t es = f32 ? sizeof(float) : sizeof(double);  // state element size of the forward
    AdjRecorder rec;
    rec.c = c;
    rec.s = c->stream;
    rec.f32 = f32;
    try {
        if (f32 && !c->shadow) make_shadow(c);
        hlbm_ctx *tc = f32 ? c->shadow : c;
        if (!tc->adj.built) build_adjoint_tables(tc);
        if (!tc->adj.coupled_built) build_coupled_tables(tc);
        const AdjTables &A = tc->adj;
        const DevCtx DT = tc->dev;  // FP64 tables of the reverse sweep (D0 itself for FP64)
        cudaStream_t s = c->stream;
        const int Np = D0.m.Np, nr = std::max(1, D0.m.n_ring);
        const size_t plane = size_t(9) * Np, qn = size_t(12) * nr;
        auto copy = [&](void *dst, const void *src, size_t elems) {  // forward state (es bytes per element)
            ck(cudaMemcpyAsync(dst, src, elems * es, cudaMemcpyDeviceToDevice, s), "copy");
        };
        auto copyd = [&](double *dst, const double *src, size_t doubles) {
            ck(cudaMemcpyAsync(dst, src, doubles * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
        };
        // the evolving state: every level's lattice and band buffers, the mesh
        // buffers and the interface-data buffers (a "snapshot" copies all)
        std::vector<std::pair<void **, size_t>> parts;  // (buffer in W, doubles)
        DevCtx W = D0;
        for (int l = 0; l < L; l++) {
            parts.push_back({&W.lv[l].f, 9 * D0.lv[l].stride});
            if (D0.lv[l].has_child)
                for (int b = 0; b < 2; b++) parts.push_back({&W.lv[l].snap[b], 12 * size_t(D0.lv[l].band_n)});
        }
        for (int b = 0; b < 2; b++) {
            parts.push_back({&W.m.g[b], plane});
            parts.push_back({&W.m.Qb[b], qn});
        }
        size_t state_doubles = 0;
        for (auto &pt : parts) state_doubles += pt.second;
        const void *orig[64];
        for (size_t k = 0; k < parts.size(); k++) {
            orig[k] = *parts[k].first;
            *parts[k].first = scr(parts[k].second * es);
            copy(*parts[k].first, orig[k], parts[k].second);
        }
        auto save = [&](double *dst_) {
            char *dst = (char *)dst_;
            for (auto &pt : parts) {
                copy(dst, *pt.first, pt.second);
                dst += pt.second * es;
            }
        };
        auto load = [&](const double *src_) {
            const char *src = (const char *)src_;
            for (auto &pt : parts) {
                copy(*pt.first, src, pt.second);
                src += pt.second * es;
            }
        };
        W.force_cap = K;
        W.force_buf = scr(2 * size_t(K) * sizeof(double));
        W.force_partial = scr(2 * size_t(std::max(1, (D0.m.n_edges + 127) / 128)) * sizeof(double));
        W.force_counter = (int *)scr(2 * sizeof(int));
        W.flag = W.force_counter + 1;
        ck(cudaMemsetAsync(W.force_counter, 0, 2 * sizeof(int), s), "memset");
        W.m.wall_stats = 0;
        auto phase = [&](long k) {
            std::swap(c->dev, W);
            set_phase(c, k0 + k);
            std::swap(c->dev, W);
        };
        auto step = [&]() {
            std::swap(c->dev, W);
            try {
                if (f32) coarse_step<float, float>(c, s);
                else coarse_step<double, double>(c, s);
            } catch (...) {
                std::swap(c->dev, W);
                throw;
            }
            std::swap(c->dev, W);
        };
        // Recomputation checkpointing: segments of S = ceil(sqrt(K)) coarse
        // steps; the first pass keeps the state at each segment start, the
        // reverse sweep re-runs one segment at a time keeping its step starts,
        // and re-runs each step once more while recording it.
        const int S = std::max(1, int(std::ceil(std::sqrt(double(K)))));
        const int nseg = (K + S - 1) / S;
        std::vector<double *> cpt(nseg), sst(S);
        for (int j = 0; j < nseg; j++) cpt[j] = scr(state_doubles * es);
        for (int j = 0; j < S; j++) sst[j] = scr(state_doubles * es);
        for (int k = 0; k < K; k++) {  // first pass: forces and segment checkpoints
            phase(k);
            if (k % S == 0) save(cpt[k / S]);
            step();
        }
        ck(cudaGetLastError(), "forward steps");
        std::vector<double> fb(2 * size_t(K));
        ck(cudaMemcpyAsync(fb.data(), W.force_buf, fb.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
        int flag = 0;
        ck(cudaMemcpyAsync(&flag, W.flag, sizeof(int), cudaMemcpyDeviceToHost, s), "D2H");
        // ---- reverse sweep: cotangents of every level's lattice (AA slots),
        // of the band data of levels with a child, of the mesh state and of
        // the interface data of the finest step being reversed
        std::vector<double *> lam_f(L), lsA(L, nullptr), lsB(L, nullptr);
        size_t maxper = 1;
        for (int l = 0; l < L; l++) {
            const DevLevel &dl = D0.lv[l];
            lam_f[l] = scr(9 * dl.stride * sizeof(double));
            ck(cudaMemsetAsync(lam_f[l], 0, 9 * dl.stride * sizeof(double), s), "memset");
            if (dl.has_child) {
                lsA[l] = scr(12 * size_t(dl.band_n) * sizeof(double));
                lsB[l] = scr(12 * size_t(dl.band_n) * sizeof(double));
                ck(cudaMemsetAsync(lsA[l], 0, 12 * size_t(dl.band_n) * sizeof(double), s), "memset");
                ck(cudaMemsetAsync(lsB[l], 0, 12 * size_t(dl.band_n) * sizeof(double), s), "memset");
            }
            if (l > 0) maxper = std::max(maxper, size_t(2 * dl.nx + 2 * (dl.ny - 2)));
        }
        double *lam_g = scr(plane * sizeof(double)), *lam_t = scr(plane * sizeof(double));
        double *lQ0 = scr(qn * sizeof(double)), *lQ1 = scr(qn * sizeof(double)), *qtmp = scr(qn * sizeof(double));
        double *lamq = scr(12 * size_t(std::max(1, D0.m.n_is)) * sizeof(double));
        double *lamp = scr(12 * maxper * sizeof(double));
        double *st = scr((size_t(ns) + 1) * plane * sizeof(double));
        double *gc = scr(std::max<size_t>(1, 3 * P.col.size()) * sizeof(double));
        double *rs = scr(3 * plane * sizeof(double));
        double *gg = scr(9 * size_t(n) * sizeof(double));
        double *gl = grad_lattice ? scr(lat_total * sizeof(double)) : nullptr;
        // geometry cotangents accumulated over the steps: Eq. 3 entries (gc),
        // wall-edge normals, Eq. 8 and Eq. 9 weights
        const size_t nis = size_t(std::max(1, D0.m.n_is)), nwe = size_t(std::max(1, D0.m.n_edges));
        double *hacc = geo ? scr(2 * nwe * sizeof(double)) : nullptr;
        double *lw6 = geo ? scr(6 * nis * sizeof(double)) : nullptr;
        double *lw9 = geo ? scr(9 * size_t(nr) * sizeof(double)) : nullptr;
        double *gxy = grad_xy ? scr(2 * size_t(n) * sizeof(double)) : nullptr;
        double *gsc = geo ? scr((3 * size_t(n) + 6 * nis) * sizeof(double)) : nullptr;
        double *daoa = scr(sizeof(double));
        ck(cudaMemsetAsync(gc, 0, std::max<size_t>(1, 3 * P.col.size()) * sizeof(double), s), "memset");
        if (geo) {
            ck(cudaMemsetAsync(hacc, 0, 2 * nwe * sizeof(double), s), "memset");
            ck(cudaMemsetAsync(lw6, 0, 6 * nis * sizeof(double), s), "memset");
            ck(cudaMemsetAsync(lw9, 0, 9 * size_t(nr) * sizeof(double), s), "memset");
        }
        ck(cudaMemsetAsync(lam_g, 0, plane * sizeof(double), s), "memset");
        ck(cudaMemsetAsync(st, 0, (size_t(ns) + 1) * plane * sizeof(double), s), "memset");
        ck(cudaMemsetAsync(lQ0, 0, qn * sizeof(double), s), "memset");
        ck(cudaMemsetAsync(lQ1, 0, qn * sizeof(double), s), "memset");
        const int fin = L - 1;
        const double inv_q = 1.0 / P.qdyn, dt = 1.0 / ns, dt_tau = dt / P.tau_u, csP = dt_tau * (11.0 / 18.0);
        const double scale5 = 1.0 - 1.0 / (2.0 * D0.lv[fin].tau);
        const double *ring_w = (const double *)DT.m.ring_w;
        std::vector<size_t> subtree(L, 1);  // level steps in one advance() of level l
        for (int l = L - 2; l >= 0; l--) subtree[l] = 1 + 2 * subtree[l + 1];
        bool terminal = false;
        // reverse of one level step (the forward's order: hole nodes, collision,
        // boundary ring, interface data and finite-volume group)
        auto level_adj = [&](const LevelRec &R) {
            const int l = R.l, Pk = R.P;
            const DevLevel &dl = DT.lv[l];
            if (l == fin) {
                DevCtx V = DT;  // the finite-volume group again (FP64), from the step's records
                V.lv[l].f = R.f_end;
                V.lv[l].parity = Pk ^ 1;
                V.m.Q0 = R.Q0;
                V.m.Q1 = qtmp;
                copyd(st, R.g_start, plane);
                V.m.g[0] = st;
                V.m.gcur = 0;
                launch_ring_interp<double, double>(V, true, s);  // interface rows at theta = 0
                V.m.Q1 = R.Q1;
                for (int m = 0; m < ns; m++) {
                    V.m.g[0] = st + size_t(m) * plane;
                    V.m.g[1] = st + size_t(m + 1) * plane;
                    launch_fv<double, double>(V, m, s);
                }
                if (terminal) {  // the coarse step's force sample
                    launch_adj_terminal(A, st + size_t(ns) * plane, Np, n, wd * wavg, wl * wavg, inv_q, lam_g, s, true);
                    if (geo)
                        launch_adj_wall_normal(A, st + size_t(ns) * plane, Np, wd * wavg, wl * wavg, inv_q, hacc, s);
                    terminal = false;
                }
                double *lin = lam_g, *lout = lam_t;
                for (int m = ns - 1; m >= 0; m--) {
                    const double th = double(m + 1) / ns;
                    if (m < ns - 1) launch_adj_ring_rows(DT.m, scale5, 1.0 - th, th, lin, lQ0, lQ1, s);
                    launch_fv_adjoint(A, st + size_t(m) * plane, Np, n, csP, P.n_wall, P.ring_start,
                                      m < ns - 1 ? 1 : 0, dt, dt_tau, lin, lout, gc, rs, s);
                    std::swap(lin, lout);
                }
                launch_adj_ring_rows(DT.m, scale5, 1.0, 0.0, lin, lQ0, lQ1, s);
                if (lin != lam_g) std::swap(lam_g, lam_t);
                if (geo) launch_adj_ring_weights(dl, DT.m, R.f_end, Pk ^ 1, lQ1, lw9, s);
                launch_adj_ring_lattice(dl, R.f_end, Pk ^ 1, A, ring_w, lQ1, DT.m.n_ring, lam_f[l], s);
            }
            if (l == 0) launch_adj_outer_bc(dl, R.f_end, Pk ^ 1, P.u0, lam_f[0], s);
            else
                launch_adj_prolong(DT.lv[l - 1], dl, Pk ^ 1, R.theta, R.sA, R.sB, A.pp[l], A.pk[l], A.pw[l], lam_f[l],
                                   lamp, lsA[l - 1], lsB[l - 1], s);
            launch_adj_collide(dl, R.f_start, Pk, lam_f[l], s);
            if (l == fin) {
                launch_adj_hole(dl, DT.m, A, R.g_start, Pk, lam_f[l], lamq, lam_g, s, lw6);
                if (geo) launch_adj_ring_weights(dl, DT.m, R.f_start, Pk, lQ0, lw9, s);
                launch_adj_ring_lattice(dl, R.f_start, Pk, A, ring_w, lQ0, DT.m.n_ring, lam_f[l], s);
                ck(cudaMemsetAsync(lQ0, 0, qn * sizeof(double), s), "memset");
                ck(cudaMemsetAsync(lQ1, 0, qn * sizeof(double), s), "memset");
            }
        };
        // reverse of advance(l) whose level step is record idx: restriction,
        // the two child steps (second first), band after the step, the level
        // step, band at the step start
        std::function<void(size_t, int)> rev = [&](size_t idx, int l) {
            const LevelRec R = rec.recs[idx];
            if (l < L - 1) {
                const size_t second = idx + 1 + subtree[l + 1];
                const LevelRec &R2 = rec.recs[second];
                launch_adj_restrict(DT.lv[l], DT.lv[l + 1], R.P ^ 1, R2.P ^ 1, R.f_child, lam_f[l], lam_f[l + 1], s);
                rev(second, l + 1);
                rev(idx + 1, l + 1);
                launch_adj_snapshot(DT.lv[l], R.f_end, R.P ^ 1, lsB[l], lam_f[l], s);
                ck(cudaMemsetAsync(lsB[l], 0, 12 * size_t(D0.lv[l].band_n) * sizeof(double), s), "memset");
            }
            level_adj(R);
            if (l < L - 1) {
                launch_adj_snapshot(DT.lv[l], R.f_start, R.P, lsA[l], lam_f[l], s);
                ck(cudaMemsetAsync(lsA[l], 0, 12 * size_t(D0.lv[l].band_n) * sizeof(double), s), "memset");
            }
        };
        for (int k = K - 1; k >= 0; k--) {
            const int j = k / S, ka = j * S;
            if (k == std::min(K, ka + S) - 1) {  // re-run segment j keeping its step starts
                phase(ka);
                load(cpt[j]);
                for (int kk = ka; kk <= k; kk++) {
                    phase(kk);
                    save(sst[kk - ka]);
                    if (kk < k) step();
                }
            }
            // step k once more, recorded (one stream: no side branches)
            phase(k);
            load(sst[k - ka]);
            std::fill(c->side_ok, c->side_ok + hlbm::kMaxLevels, false);
            c->rec = &rec;
            try {
                step();
            } catch (...) {
                c->rec = nullptr;
                throw;
            }
            c->rec = nullptr;
            std::copy(side0, side0 + hlbm::kMaxLevels, c->side_ok);
            if (rec.recs.size() != subtree[0]) throw CudaError{"unexpected level-step count in the recorded step"};
            terminal = k >= n_skip;  // the step's force sample is averaged
            rev(0, 0);
            ck(cudaStreamSynchronize(s), "sync");  // the records are freed next
            rec.release();
        }
        // gradients with respect to the state at the first step: every level's
        // populations (level order) and the mesh populations
        phase(0);
        load(sst[0]);
        if (gl) {
            size_t off = 0;
            for (int l = 0; l < L; l++) {
                const DevLevel &dl = DT.lv[l];
                launch_adj_lattice_out(dl, lam_f[l], l == 0 ? int(k0 & 1) : 0, gl + off, s);
                off += 9 * size_t(dl.nx) * dl.ny;
            }
        }
        const double *g0 = (const double *)W.m.g[W.m.gcur];
        if (f32) {  // the initial mesh state, widened
            double *g64 = scr(plane * sizeof(double));
            launch_widen((const float *)W.m.g[W.m.gcur], g64, plane, s);
            g0 = g64;
        }
        launch_adj_populations(A, g0, Np, n, lam_g, gg, s);
        if (geo) {
            const double al = P.aoa_deg * M_PI / 180.0;
            launch_adj_geometry_coupled(A, DT.m, n, gc, hacc, lw6, lw9, std::cos(al), std::sin(al), P.pivot[0],
                                        P.pivot[1], gsc, gxy, daoa, s);
        }
        ck(cudaGetLastError(), "adjoint kernels");
        if (grad_xy) ck(cudaMemcpyAsync(grad_xy, gxy, 2 * size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
        if (dJ_daoa) ck(cudaMemcpyAsync(dJ_daoa, daoa, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
        if (gl) ck(cudaMemcpyAsync(grad_lattice, gl, lat_total * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
        if (grad_mesh) ck(cudaMemcpyAsync(grad_mesh, gg, 9 * size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
        ck(cudaStreamSynchronize(s), "sync");
        double jsum = 0.0;
        for (int k = n_skip; k < K; k++) jsum += wd * fb[2 * size_t(k)] + wl * fb[2 * size_t(k) + 1];
        *J = jsum * wavg;
        if (flag & 2) rc = fail(c, HLBM_ETIMEOUT, "a device-side wait gave up (operator copy did not arrive)");
        else if (flag) rc = fail(c, HLBM_EUNSTABLE, "NaN in the force reduction of the forward steps");
    } catch (const CudaError &e) {
        rc = fail(c, HLBM_ECUDA, e.msg);
    } catch (const std::bad_alloc &) {
        rc = fail(c, HLBM_ENOMEM, "host allocation failed");
    }
    c->rec = nullptr;
    cudaStreamSynchronize(c->stream);
    rec.release();
    c->dev = D0;
    std::copy(side0, side0 + hlbm::kMaxLevels, c->side_ok);
    c->launches = launches0;
    c->launches_per_step = lps0;
    for (void *p : scratch) dfree(c, p);
    return rc;
}

int hlbm_wall_stats_reset(hlbm_ctx *c)
{
    if (!c) return HLBM_EINVAL;
    const DevMesh &M = c->dev.m;
    if (!M.wall_stats) return fail(c, HLBM_ESTATE, "the context was created without wall_stats");
    if (c->plan.n_wall > 0) {
        cudaError_t e = cudaMemsetAsync(M.wall_acc, 0, 3 * size_t(c->plan.n_wall) * sizeof(double), c->stream);
        if (e != cudaSuccess) return fail(c, HLBM_ECUDA, cudaGetErrorString(e));
    }
    c->stats_base = c->steps;
    return HLBM_OK;
}

// ------------------------------------------------------------- checkpoint ----
// File: "HLBMCKPT", uint32 header length, JSON header, then the device buffers
// as raw bytes in the order of ckpt_buffers (sizes in the header).
namespace {

struct Blob {
    void *ptr;
    size_t bytes;
};

std::vector<Blob> ckpt_buffers(hlbm_ctx *c)
{
    const DevCtx &D = c->dev;
    const int p = c->plan.precision;
    const size_t sz = p == HLBM_FP64 ? 8 : (p == HLBM_FP32 ? 4 : 2);  // lattice storage
    const size_t tz = p == HLBM_FP64 ? 8 : 4;                         // mesh and interface data
    std::vector<Blob> v;
    for (int l = 0; l < D.L; l++) {
        const DevLevel &dl = D.lv[l];
        v.push_back({dl.f, 9 * dl.stride * sz});
        if (dl.snap[0]) {
            v.push_back({dl.snap[0], 12 * size_t(dl.band_n) * tz});
            v.push_back({dl.snap[1], 12 * size_t(dl.band_n) * tz});
        }
    }
    const DevMesh &m = D.m;
    if (m.n > 0) {
        v.push_back({m.g[m.gcur], 9 * size_t(m.Np) * tz});
        const size_t qn = 12 * size_t(std::max(1, m.n_ring)) * tz;
        v.push_back({m.Qb[0], qn});
        v.push_back({m.Qb[1], qn});
        if (m.wall_stats && m.wall_acc) v.push_back({m.wall_acc, 3 * size_t(c->plan.n_wall) * sizeof(double)});
    }
    if (D.force_buf) {
        v.push_back({D.force_buf, 2 * size_t(D.force_cap) * sizeof(double)});
        v.push_back({D.force_counter, 2 * sizeof(int)});
    }
    return v;
}

std::string ckpt_header(hlbm_ctx *c, const std::vector<Blob> &v)
{
    const Plan &P = c->plan;
    std::string h = "{\"version\": 1, \"precision\": " + std::to_string(P.precision) + ", \"levels\": [";
    for (int l = 0; l < P.L; l++)
        h += std::string(l ? ", " : "") + "[" + std::to_string(P.lv[l].nx) + ", " + std::to_string(P.lv[l].ny) + ", " +
             std::to_string(P.lv[l].ox) + ", " + std::to_string(P.lv[l].oy) + "]";
    h += "], \"mesh_nodes\": " + std::to_string(P.n) + ", \"n_sub\": " + std::to_string(P.n_sub) +
         ", \"force_cap\": " + std::to_string(c->dev.force_cap) + ", \"wall_stats\": " +
         std::to_string(c->dev.m.wall_stats) + ", \"fv_filter\": " + std::to_string(c->dev.fv_filter) +
         ", \"buffers\": [";
    for (size_t k = 0; k < v.size(); k++) h += std::string(k ? ", " : "") + std::to_string(v[k].bytes);
    h += "]}";
    return h;
}

// the part of the header that must match the loading context (everything
// before the mutable counters)
std::string ckpt_counters(hlbm_ctx *c)
{
    char buf[256];
    std::snprintf(buf, sizeof buf, "%ld %ld %ld %.17g", c->steps, c->forces_read, c->stats_base, c->mass0);
    return buf;
}

}  // namespace

int hlbm_save(hlbm_ctx *c, const char *path)
{
    if (!c || !path) return c ? fail(c, HLBM_EINVAL, "path is NULL") : HLBM_EINVAL;
    if (c->timing_dirty) return fail(c, HLBM_ESTATE, "the state was consumed by hlbm_time_kernel");
    std::vector<Blob> v = ckpt_buffers(c);
    std::string head = ckpt_header(c, v), cnt = ckpt_counters(c);
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return fail(c, HLBM_EINVAL, std::string("cannot open ") + path + " for writing");
    bool ok = true;
    try {
        ck(cudaStreamSynchronize(c->stream), "sync");
        const uint32_t hl = uint32_t(head.size()), cl = uint32_t(cnt.size());
        ok = std::fwrite("HLBMCKPT", 1, 8, fp) == 8 && std::fwrite(&hl, 4, 1, fp) == 1 &&
             std::fwrite(head.data(), 1, hl, fp) == hl && std::fwrite(&cl, 4, 1, fp) == 1 &&
             std::fwrite(cnt.data(), 1, cl, fp) == cl;
        std::vector<char> host;
        for (const Blob &b : v) {
            if (!ok) break;
            host.resize(b.bytes);
            ck(cudaMemcpy(host.data(), b.ptr, b.bytes, cudaMemcpyDeviceToHost), "D2H");
            ok = std::fwrite(host.data(), 1, b.bytes, fp) == b.bytes;
        }
    } catch (const CudaError &e) {
        std::fclose(fp);
        return fail(c, HLBM_ECUDA, e.msg);
    }
    if (std::fclose(fp) != 0) ok = false;
    return ok ? HLBM_OK : fail(c, HLBM_EINVAL, std::string("writing ") + path + " failed");
}

int hlbm_load(hlbm_ctx *c, const char *path)
{
    if (!c || !path) return c ? fail(c, HLBM_EINVAL, "path is NULL") : HLBM_EINVAL;
    std::vector<Blob> v = ckpt_buffers(c);
    const std::string want = ckpt_header(c, v);
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return fail(c, HLBM_EINVAL, std::string("cannot open ") + path);
    auto bad = [&](const std::string &msg) {
        std::fclose(fp);
        return fail(c, HLBM_EINVAL, msg);
    };
    char magic[8];
    uint32_t hl = 0, cl = 0;
    if (std::fread(magic, 1, 8, fp) != 8 || std::memcmp(magic, "HLBMCKPT", 8) != 0) return bad("not a checkpoint");
    if (std::fread(&hl, 4, 1, fp) != 1 || hl > (1u << 20)) return bad("bad checkpoint header");
    std::string head(hl, '\0');
    if (std::fread(&head[0], 1, hl, fp) != hl) return bad("truncated checkpoint header");
    if (head != want) return bad("checkpoint of another configuration: " + head);
    if (std::fread(&cl, 4, 1, fp) != 1 || cl > 255) return bad("bad checkpoint counters");
    std::string cnt(cl, '\0');
    if (std::fread(&cnt[0], 1, cl, fp) != cl) return bad("truncated checkpoint counters");
    long steps = 0, forces_read = 0, stats_base = 0;
    double mass0 = 0.0;
    if (std::sscanf(cnt.c_str(), "%ld %ld %ld %lg", &steps, &forces_read, &stats_base, &mass0) != 4 || steps < 0)
        return bad("bad checkpoint counters");
    // the current mesh buffer depends on the step count: point the blob list at it
    set_phase(c, steps);
    v = ckpt_buffers(c);
    std::vector<char> host;
    try {
        ck(cudaStreamSynchronize(c->stream), "sync");
        for (const Blob &b : v) {
            host.resize(b.bytes);
            if (std::fread(host.data(), 1, b.bytes, fp) != b.bytes) {
                set_phase(c, c->steps);
                return bad("truncated checkpoint data");
            }
            ck(cudaMemcpy(b.ptr, host.data(), b.bytes, cudaMemcpyHostToDevice), "H2D");
        }
    } catch (const CudaError &e) {
        std::fclose(fp);
        return fail(c, HLBM_ECUDA, e.msg);
    }
    std::fclose(fp);
    c->steps = steps;
    c->forces_read = forces_read;
    c->stats_base = stats_base;
    c->mass0 = mass0;
    c->timing_dirty = false;
    return HLBM_OK;
}

static void batch_release(hlbm_batch *b)
{
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (int k = 0; k < 2; k++)
        if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
    for (cudaEvent_t e : b->ready)
        if (e) cudaEventDestroy(e);
    if (b->done) cudaEventDestroy(b->done);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

int hlbm_batch_create(hlbm_ctx *const *ctxs, int n, void *stream, hlbm_batch **out)
{
    if (!out) return fail(nullptr, HLBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ctxs || n < 1) return fail(nullptr, HLBM_EINVAL, "a batch needs at least one context");
    for (int i = 0; i < n; i++) {
        hlbm_ctx *c = ctxs[i];
        if (!c) return fail(nullptr, HLBM_EINVAL, "context " + std::to_string(i) + " is NULL");
        if (!c->use_graphs || !c->graph_tmpl[0] || !c->graph_tmpl[1])
            return fail(nullptr, HLBM_EINVAL, "context " + std::to_string(i) + " was created without CUDA graphs");
        if (c->timing_dirty)
            return fail(nullptr, HLBM_ESTATE, "context " + std::to_string(i) + " was consumed by hlbm_time_kernel");
        for (int j = 0; j < i; j++)
            if (ctxs[j] == c) return fail(nullptr, HLBM_EINVAL, "context " + std::to_string(i) + " appears twice");
    }
    hlbm_batch *b = new hlbm_batch();
    cudaGraph_t g = nullptr;
    try {
        b->ctx.assign(ctxs, ctxs + n);
        for (hlbm_ctx *c : b->ctx) {
            b->base.push_back(c->steps);
            cudaEvent_t e = nullptr;
            ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
            b->ready.push_back(e);
        }
        ck(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming), "event");
        if (stream) {
            b->stream = static_cast<cudaStream_t>(stream);
        } else {
            ck(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "stream");
            b->own_stream = true;
        }
        // graph k: every context's coarse-step graph for its phase after k
        // batch steps, as child graphs with no edges between them
        for (int k = 0; k < 2; k++) {
            ck(cudaGraphCreate(&g, 0), "graph create");
            for (hlbm_ctx *c : b->ctx) {
                cudaGraphNode_t node = nullptr;
                ck(cudaGraphAddChildGraphNode(&node, g, nullptr, 0, c->graph_tmpl[(c->steps + k) & 1]), "child graph");
            }
            ck(cudaGraphInstantiate(&b->exec[k], g, 0), "graph instantiate");
            cudaGraphDestroy(g);
            g = nullptr;
        }
    } catch (const CudaError &e) {
        if (g) cudaGraphDestroy(g);
        batch_release(b);
        delete b;
        return fail(nullptr, HLBM_ECUDA, e.msg);
    }
    *out = b;
    return HLBM_OK;
}

int hlbm_batch_step(hlbm_batch *b, int n_coarse)
{
    if (!b) return HLBM_EINVAL;
    if (n_coarse < 0) { b->err = "n_coarse must be >= 0"; return HLBM_EINVAL; }
    for (size_t i = 0; i < b->ctx.size(); i++) {
        hlbm_ctx *c = b->ctx[i];
        if (c->timing_dirty || c->steps != b->base[i] + b->steps) {
            b->err = "context " + std::to_string(i) + " was advanced or consumed outside the batch";
            return HLBM_ESTATE;
        }
    }
    bool check = false;
    Range r("hlbm_batch_step");
    try {
        // the batch stream waits for whatever the contexts' own streams hold
        for (size_t i = 0; i < b->ctx.size(); i++) {
            ck(cudaEventRecord(b->ready[i], b->ctx[i]->stream), "event record");
            ck(cudaStreamWaitEvent(b->stream, b->ready[i], 0), "stream wait");
        }
        for (int k = 0; k < n_coarse; k++) {
            ck(cudaGraphLaunch(b->exec[b->steps & 1], b->stream), "graph launch");
            b->steps++;
            for (hlbm_ctx *c : b->ctx) {
                c->steps++;
                set_phase(c, c->steps);
                if (c->check_every > 0 && (c->steps % c->check_every) == 0) check = true;
            }
        }
        // later work on a context's own stream (readback, hlbm_step) follows the batch
        ck(cudaEventRecord(b->done, b->stream), "event record");
        for (hlbm_ctx *c : b->ctx) ck(cudaStreamWaitEvent(c->stream, b->done, 0), "stream wait");
        if (check) {
            ck(cudaStreamSynchronize(b->stream), "sync");
            for (size_t i = 0; i < b->ctx.size(); i++) {
                int flag = 0;
                ck(cudaMemcpy(&flag, b->ctx[i]->dev.flag, sizeof(int), cudaMemcpyDeviceToHost), "flag");
                if (flag & 2) {
                    b->err = "case " + std::to_string(i) + ": a device-side wait gave up";
                    return HLBM_ETIMEOUT;
                }
                if (flag) {
                    b->err = "case " + std::to_string(i) + ": NaN in the force reduction (unstable)";
                    return HLBM_EUNSTABLE;
                }
                hlbm_ctx *c = b->ctx[i];
                c->mass_drift = std::fabs(level0_mass(c) - c->mass0) / c->mass0;
                if (!(c->mass_drift <= kMassDriftLimit)) {
                    b->err = "case " + std::to_string(i) + ": total mass drifted by " + std::to_string(c->mass_drift);
                    return HLBM_EUNSTABLE;
                }
            }
        }
    } catch (const CudaError &e) {
        b->err = e.msg;
        return HLBM_ECUDA;
    }
    return HLBM_OK;
}

int hlbm_batch_sync(hlbm_batch *b)
{
    if (!b) return HLBM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) { b->err = cudaGetErrorString(e); return HLBM_ECUDA; }
    return HLBM_OK;
}

const char *hlbm_batch_last_error(const hlbm_batch *b) { return b ? b->err.c_str() : g_create_err.c_str(); }

int hlbm_batch_destroy(hlbm_batch *b)
{
    if (!b) return HLBM_OK;
    batch_release(b);
    delete b;
    return HLBM_OK;
}

const char *hlbm_last_error(const hlbm_ctx *c)
{
    if (!c) return g_create_err.c_str();
    return c->err.c_str();
}

}  // extern "C"
