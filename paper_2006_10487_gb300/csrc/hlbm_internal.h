// Internal declarations of the HLBM library (host set-up plan, device state,
// kernel launchers).  Not part of the public ABI.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <functional>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hlbm.h"

namespace hlbm {

constexpr int kMaxLevels = 8;
constexpr int kMeshGrid = 63;  // grid id of the mesh in the initial-state generator

// Host-side description of one Cartesian level.
struct LevelPlan {
    int nx = 0, ny = 0, ox = 0, oy = 0;
    double tau = 0.0;
    // finest level with a mesh: per row y, nodes x in [hx0[y], hx1[y]) are not computed
    std::vector<int> hx0, hx1;
    // refinement towards the child level (if any)
    bool has_child = false;
    int cmx = 0, cmy = 0;  // child box size in this level's cells
    int cox = 0, coy = 0;  // child origin in this level's nodes
};

// Everything hlbm_create derives on the host, in FP64.
struct Plan {
    int L = 0;
    LevelPlan lv[kMaxLevels];
    double u0 = 0, nu = 0, tau_u = 0, chord = 0, qdyn = 0;
    double aoa_deg = 0, pivot[2] = {0, 0};  // mesh pose: rotation by -aoa about the pivot
    int n_sub = 0;
    int precision = HLBM_FP64;
    uint64_t seed = 0;
    double perturb = 0;

    // mesh, input node order
    int n = 0, ntri = 0;
    std::vector<double> xy;       // rotated coordinates [n][2]
    std::vector<int> tri;         // [ntri][3]
    std::vector<uint8_t> kind;    // [n]
    std::vector<int> rowptr, col; // Eq. 3 operators, CSR, columns ascending
    std::vector<double> sx, sy, cc, area;
    // device order: wall nodes, then fluid nodes, then ring nodes (stable)
    std::vector<int> perm;  // perm[new] = old
    std::vector<int> inv;   // inv[old] = new
    int n_wall = 0, ring_start = 0, n_ring = 0;
    // structured interpolation nodes (Eq. 4, Eq. 8)
    std::vector<int> is_node;    // finest-level node index y*nx + x, row-major
    std::vector<int> is_don;     // [n_is][6] mesh nodes (input order)
    std::vector<double> is_w;    // [n_is][6]
    // unstructured interpolation nodes (Eq. 5, Eq. 9), ring nodes in input order
    std::vector<int> ring;       // mesh node (input order)
    std::vector<int> ring_don;   // [n_ring][9] finest-level node index y*nx + x
    std::vector<double> ring_w;  // [n_ring][9]
    // wall edges (a -> b, fluid on the left), input order
    std::vector<int> wea, web;
    // wall nodes (ascending input index = device rows 0 .. n_wall-1):
    // [n_wall][7] = x/C, side, |N_P|, n_x, n_y, s_x, s_y (Eq. 12-13)
    std::vector<double> wall_geo;
};

// Builds the plan; returns HLBM_OK or an error code with a message in err.
int build_plan(const hlbm_level *lv, int n_levels, const hlbm_mesh *m, double Re, double Ma,
               double aoa_deg, const hlbm_options *opt, Plan &plan, std::string &err);

// splitmix64-based initial density deviate in [-1, 1) (host side).
double init_deviate(uint64_t seed, uint64_t grid, uint64_t node);

// Runs task(j) for j in [0, n_tasks) on the process's host worker threads
// (up to 15, started on first use and kept) and the calling thread, and
// returns when all have run; false if a task threw (every task still runs).
// Calls from different threads take turns; a call made from inside a task, or
// in a process forked after the workers started, runs its tasks inline.
bool run_tasks(int n_tasks, const std::function<void(int)> &task);

// Runs f(begin, end) over [0, n) in contiguous chunks of at least `grain`
// items on up to 16 host threads (inline when there is one chunk).  Chunks
// write disjoint outputs, so results do not depend on the thread count.  A
// chunk that throws makes the call throw std::bad_alloc after all have ended.
template <typename F> void parallel_for(int n, F f, int grain = 2048)
{
    const int hw = int(std::max(1u, std::thread::hardware_concurrency()));
    const int nt = std::min(std::min(hw, 16), std::max(1, n / std::max(1, grain)));
    if (nt <= 1) {
        f(0, n);
        return;
    }
    const bool ok = run_tasks(nt, [&](int j) { f(int(long(n) * j / nt), int(long(n) * (j + 1) / nt)); });
    if (!ok) throw std::bad_alloc();
}

// Message returned by hlbm_last_error(NULL) on this thread.
void set_thread_error(const std::string &msg);

}  // namespace hlbm
