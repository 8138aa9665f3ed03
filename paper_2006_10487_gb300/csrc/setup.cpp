// Host set-up of the HLBM step: geometry, Eq. 3 finite-volume operators,
// Eq. 8 / Eq. 9 interpolation stencils, refinement maps and the sub-step
// count.  All in FP64; the device tables are converted from this plan.
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstring>

#include "hlbm_internal.h"

namespace hlbm {
namespace {

struct V2 {
    double x, y;
};
inline V2 sub(V2 a, V2 b) { return {a.x - b.x, a.y - b.y}; }
// outward normal times length of a directed segment along d (domain on the left)
inline V2 perp(V2 d) { return {d.y, -d.x}; }


// Solves A x = b for a small dense system by Gauss-Jordan elimination with
// full pivoting; A is row-major n x n.  Returns false if singular.
bool gauss_jordan(int n, double *A, double *b)
{
    int colmap[16];
    for (int i = 0; i < n; i++) colmap[i] = i;
    for (int k = 0; k < n; k++) {
        int pr = k, pc = k;
        double best = 0.0;
        for (int r = k; r < n; r++)
            for (int c = k; c < n; c++)
                if (std::fabs(A[r * n + c]) > best) { best = std::fabs(A[r * n + c]); pr = r; pc = c; }
        if (best == 0.0) return false;
        if (pr != k) {
            for (int c = 0; c < n; c++) std::swap(A[k * n + c], A[pr * n + c]);
            std::swap(b[k], b[pr]);
        }
        if (pc != k) {
            for (int r = 0; r < n; r++) std::swap(A[r * n + k], A[r * n + pc]);
            std::swap(colmap[k], colmap[pc]);
        }
        double inv = 1.0 / A[k * n + k];
        for (int c = 0; c < n; c++) A[k * n + c] *= inv;
        b[k] *= inv;
        for (int r = 0; r < n; r++) {
            if (r == k) continue;
            double m = A[r * n + k];
            if (m == 0.0) continue;
            for (int c = 0; c < n; c++) A[r * n + c] -= m * A[k * n + c];
            b[r] -= m * b[k];
        }
    }
    double x[16];
    for (int k = 0; k < n; k++) x[colmap[k]] = b[k];
    for (int k = 0; k < n; k++) b[k] = x[k];
    return true;
}

}  // namespace

namespace {
// The host worker threads of run_tasks: one job at a time; a job hands out
// task indices through an atomic counter to the workers and the caller.
struct Workers {
    std::mutex run_mx;                 // one job at a time
    std::mutex mx;
    std::condition_variable wake, done;
    std::vector<std::thread> th;
    const std::function<void(int)> *task = nullptr;
    int n_tasks = 0;
    std::atomic<int> next{0};
    int busy = 0;                      // workers still inside the current job
    uint64_t job = 0;                  // job generation
    std::atomic<bool> failed{false};
    pid_t pid = 0;
};
thread_local bool t_in_task = false;

void drain(Workers &w)
{
    for (int j; (j = w.next.fetch_add(1)) < w.n_tasks;) {
        try {
            (*w.task)(j);
        } catch (...) {
            w.failed = true;
        }
    }
}

Workers *workers()
{
    static std::mutex init_mx;
    static Workers *w = nullptr;
    std::lock_guard<std::mutex> lk(init_mx);
    if (w && w->pid == getpid()) return w;
    // first use, or a forked child (whose copy has no threads): a new set,
    // the old one left as it is
    Workers *nw = new Workers();
    nw->pid = getpid();
    const int hw = int(std::max(1u, std::thread::hardware_concurrency()));
    for (int k = 1; k < std::min(hw, 16); k++) {
        try {
            nw->th.emplace_back([nw]() {
                t_in_task = true;
                uint64_t seen = 0;
                for (;;) {
                    {
                        std::unique_lock<std::mutex> lk(nw->mx);
                        nw->wake.wait(lk, [&] { return nw->job != seen; });
                        seen = nw->job;
                    }
                    drain(*nw);
                    std::lock_guard<std::mutex> lk(nw->mx);
                    if (--nw->busy == 0) nw->done.notify_all();
                }
            });
            nw->th.back().detach();
        } catch (...) {
            break;  // fewer workers
        }
    }
    w = nw;
    return w;
}
}  // namespace

bool run_tasks(int n_tasks, const std::function<void(int)> &task)
{
    Workers *w = t_in_task ? nullptr : workers();
    if (!w || w->th.empty()) {
        bool ok = true;
        for (int j = 0; j < n_tasks; j++) {
            try {
                task(j);
            } catch (...) {
                ok = false;
            }
        }
        return ok;
    }
    std::lock_guard<std::mutex> run_lk(w->run_mx);
    {
        std::lock_guard<std::mutex> lk(w->mx);
        w->task = &task;
        w->n_tasks = n_tasks;
        w->next = 0;
        w->failed = false;
        w->busy = int(w->th.size());
        w->job++;
    }
    w->wake.notify_all();
    t_in_task = true;
    drain(*w);
    t_in_task = false;
    std::unique_lock<std::mutex> lk(w->mx);
    w->done.wait(lk, [&] { return w->busy == 0; });
    return !w->failed;
}

double init_deviate(uint64_t seed, uint64_t grid, uint64_t node)
{
    // splitmix64 (Steele, Lea and Flood), one output from the given state
    uint64_t z = (seed ^ (grid << 40) ^ node) + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return double(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

int build_plan(const hlbm_level *lv, int n_levels, const hlbm_mesh *m, double Re, double Ma,
               double aoa_deg, const hlbm_options *opt, Plan &P, std::string &err)
{
    if (!lv || n_levels < 1 || n_levels > kMaxLevels) { err = "n_levels must be in 1..8"; return HLBM_EINVAL; }
    if (!m) { err = "mesh pointer is NULL"; return HLBM_EINVAL; }
    if (!(Re > 0.0) || !(Ma > 0.0)) { err = "Re and Ma must be positive"; return HLBM_EINVAL; }
    if (!std::isfinite(Re) || !std::isfinite(aoa_deg) || !(Ma < 1.0)) {
        err = "Re and the angle of attack must be finite and Ma below 1";
        return HLBM_EINVAL;
    }
    hlbm_options o{};
    if (opt) o = *opt;
    if (o.precision != HLBM_FP64 && o.precision != HLBM_FP32 && o.precision != HLBM_FP16S) {
        err = "unknown precision";
        return HLBM_EINVAL;
    }
    if (o.n_sub < 0) { err = "n_sub must be >= 0"; return HLBM_EINVAL; }
    P = Plan();
    P.L = n_levels;
    P.precision = o.precision;
    P.seed = o.seed;
    P.perturb = o.perturb;
    // the chord is the length scale of Re, also for a mesh-less channel
    P.chord = m->chord;
    if (!(m->chord > 0.0)) { err = "chord must be positive"; return HLBM_EINVAL; }
    // u0 = Ma c_s with c_s^2 = 1/3; nu = u0 C / Re (finest-level units)
    P.u0 = Ma / std::sqrt(3.0);
    P.nu = P.u0 * P.chord / Re;
    P.qdyn = 0.5 * P.u0 * P.u0 * P.chord;
    // structured viscosity nu = c_s^2 (tau - 1/2) per level in its own units,
    // unstructured nu = c_s^2 tau_u (finest units)
    for (int c = 0; c < P.L; c++) {
        LevelPlan &l = P.lv[c];
        l.nx = lv[c].nx; l.ny = lv[c].ny; l.ox = lv[c].ox; l.oy = lv[c].oy;
        if (l.nx < 4 || l.ny < 4) { err = "every level needs at least 4x4 nodes"; return HLBM_EINVAL; }
        if (c == 0 && (l.ox != 0 || l.oy != 0)) { err = "level 0 must have origin (0,0)"; return HLBM_EINVAL; }
        if (c > 0 && (l.nx % 2 == 0 || l.ny % 2 == 0)) { err = "refined levels need odd node counts"; return HLBM_EINVAL; }
        double scale = std::ldexp(1.0, P.L - 1 - c);
        l.tau = 0.5 + 3.0 * P.nu / scale;
    }
    for (int c = 1; c < P.L; c++) {
        LevelPlan &pa = P.lv[c - 1], &ch = P.lv[c];
        pa.has_child = true;
        pa.cmx = (ch.nx - 1) / 2;
        pa.cmy = (ch.ny - 1) / 2;
        pa.cox = ch.ox;
        pa.coy = ch.oy;
        if (ch.ox < 2 || ch.oy < 2 || ch.ox + pa.cmx > pa.nx - 3 || ch.oy + pa.cmy > pa.ny - 3) {
            err = "a refined box must lie at least two nodes inside its parent";
            return HLBM_EINVAL;
        }
    }
    P.tau_u = 3.0 * P.nu;

    P.n = m->n_nodes;
    P.ntri = m->n_tri;
    if (P.n == 0) { P.n_sub = 0; return HLBM_OK; }
    if (!m->xy || !m->tri || !m->kind || P.ntri < 1) { err = "mesh arrays missing"; return HLBM_EINVAL; }
    for (int k = 0; k < 2 * P.n; k++)
        if (!std::isfinite(m->xy[k])) { err = "mesh coordinates must be finite"; return HLBM_EINVAL; }
    if (!std::isfinite(m->pivot[0]) || !std::isfinite(m->pivot[1]) || !std::isfinite(m->chord)) {
        err = "pivot and chord must be finite";
        return HLBM_EINVAL;
    }
    for (int k = 0; k < 4; k++)
        if (!std::isfinite(m->hole[k])) { err = "hole ellipse must be finite"; return HLBM_EINVAL; }

    // ---- rigid rotation by -alpha about the pivot (alpha > 0: nose up)
    const double al = aoa_deg * M_PI / 180.0, ca = std::cos(al), sa = std::sin(al);
    const double px = m->pivot[0], py = m->pivot[1];
    P.aoa_deg = aoa_deg;
    P.pivot[0] = px;
    P.pivot[1] = py;
    P.xy.resize(2 * size_t(P.n));
    for (int p = 0; p < P.n; p++) {
        double dx = m->xy[2 * p] - px, dy = m->xy[2 * p + 1] - py;
        P.xy[2 * p] = px + (ca * dx + sa * dy);
        P.xy[2 * p + 1] = py + (ca * dy - sa * dx);
    }
    P.tri.assign(m->tri, m->tri + 3 * size_t(P.ntri));
    P.kind.assign(m->kind, m->kind + P.n);
    for (int t = 0; t < 3 * P.ntri; t++)
        if (P.tri[t] < 0 || P.tri[t] >= P.n) { err = "triangle index out of range"; return HLBM_EINVAL; }
    for (int p = 0; p < P.n; p++)
        if (P.kind[p] > 2) { err = "unknown node kind"; return HLBM_EINVAL; }
    auto X = [&](int p) { return V2{P.xy[2 * size_t(p)], P.xy[2 * size_t(p) + 1]}; };

    // ---- directed edges a -> b of the triangles, grouped by a, with the far
    // vertex of the triangle that owns them (each directed edge at most once)
    // (per node in ascending triangle order; etri: the triangle)
    std::vector<int> eptr(size_t(P.n) + 1, 0), edst(3 * size_t(P.ntri)), efar(3 * size_t(P.ntri)),
        etri(3 * size_t(P.ntri));
    for (int t = 0; t < 3 * P.ntri; t++) eptr[P.tri[t] + 1]++;
    for (int p = 0; p < P.n; p++) eptr[p + 1] += eptr[p];
    {
        std::vector<int> fill(eptr.begin(), eptr.end() - 1);
        for (int t = 0; t < P.ntri; t++)
            for (int a = 0; a < 3; a++) {
                const int i0 = P.tri[3 * t + a], k = fill[i0]++;
                edst[k] = P.tri[3 * t + (a + 1) % 3];
                efar[k] = P.tri[3 * t + (a + 2) % 3];
                etri[k] = t;
            }
    }
    {
        std::atomic<bool> dup{false};
        parallel_for(P.n, [&](int p0, int p1) {
            for (int p = p0; p < p1; p++)
                for (int k = eptr[p]; k < eptr[p + 1]; k++)
                    for (int j = eptr[p]; j < k; j++)
                        if (edst[j] == edst[k]) dup = true;
        });
        if (dup) { err = "mesh is not a consistently oriented manifold"; return HLBM_EINVAL; }
    }
    // far vertex of the triangle owning the directed edge a -> b, -1 if none
    auto edge_far = [&](int a, int b) {
        for (int k = eptr[a]; k < eptr[a + 1]; k++)
            if (edst[k] == b) return efar[k];
        return -1;
    };

    // ---- Eq. 3 operators (cell-vertex / median-dual control volumes,
    // piecewise-linear populations).  For triangle (P, A, B), counter-clockwise,
    // the two dual faces of P's control volume contribute, in closed form,
    //   s_P += -(5/24) perp(B - A)
    //   s_A += -(1/24) perp(4B - P - 3A)
    //   s_B += -(1/24) perp(3B + P - 4A)
    // (evaluated with P at the origin)
    // (exact integration of -(c.n) f along M_PA -> G -> M_PB); a boundary
    // edge a -> b closes the control volumes of a and b with half-edge fluxes
    //   row a: s_a += -(3/8) perp(b - a), s_b += -(1/8) perp(b - a)
    //   row b: s_b += -(3/8) perp(b - a), s_a += -(1/8) perp(b - a).
    // Collision weights are the control-volume means of the hat functions:
    //   C_PP += 11/54 |T|, C_PA, C_PB += 7/108 |T|; all rows divided by
    //   A_P = sum |T| / 3.
    // rows: the node itself and every vertex of its triangles, sorted, unique
    // (the out-edges a -> b and a -> far list them all); sizes, then columns
    auto row_of = [&](int p, std::vector<int> &row) {
        row.assign(1, p);
        for (int k = eptr[p]; k < eptr[p + 1]; k++) {
            row.push_back(edst[k]);
            row.push_back(efar[k]);
        }
        std::sort(row.begin(), row.end());
        row.erase(std::unique(row.begin(), row.end()), row.end());
    };
    P.rowptr.assign(P.n + 1, 0);
    parallel_for(P.n, [&](int p0, int p1) {
        std::vector<int> row;
        for (int p = p0; p < p1; p++) {
            row_of(p, row);
            P.rowptr[p + 1] = int(row.size());
        }
    });
    for (int p = 0; p < P.n; p++) P.rowptr[p + 1] += P.rowptr[p];
    P.col.resize(P.rowptr[P.n]);
    parallel_for(P.n, [&](int p0, int p1) {
        std::vector<int> row;
        for (int p = p0; p < p1; p++) {
            row_of(p, row);
            std::copy(row.begin(), row.end(), P.col.begin() + P.rowptr[p]);
        }
    });
    P.sx.assign(P.col.size(), 0.0);
    P.sy.assign(P.col.size(), 0.0);
    P.cc.assign(P.col.size(), 0.0);
    P.area.assign(P.n, 0.0);
    auto slot = [&](int row, int c) {
        int lo = P.rowptr[row], hi = P.rowptr[row + 1];
        return int(std::lower_bound(P.col.begin() + lo, P.col.begin() + hi, c) - P.col.begin());
    };
    std::vector<double> tarea(P.ntri);
    parallel_for(P.ntri, [&](int t0, int t1) {
        for (int t = t0; t < t1; t++) {
            V2 p0 = X(P.tri[3 * t]), p1 = X(P.tri[3 * t + 1]), p2 = X(P.tri[3 * t + 2]);
            tarea[t] = 0.5 * ((p1.x - p0.x) * (p2.y - p0.y) - (p1.y - p0.y) * (p2.x - p0.x));
        }
    });
    for (int t = 0; t < P.ntri; t++)
        if (!(tarea[t] > 0.0)) { err = "inverted or degenerate triangle"; return HLBM_EINVAL; }
    // row P gathers its triangles' terms in ascending triangle order (each
    // entry's sum runs in that order whatever the thread count)
    parallel_for(P.n, [&](int r0, int r1) {
        for (int ip = r0; ip < r1; ip++)
            for (int k = eptr[ip]; k < eptr[ip + 1]; k++) {
                const int ia = edst[k], ib = efar[k];
                const double at = tarea[etri[k]];
                // edge vectors from P (keeps the short dual segments free of
                // cancellation between large absolute coordinates)
                V2 A = sub(X(ia), X(ip)), B = sub(X(ib), X(ip));
                V2 dP = perp(sub(B, A));
                V2 dA = perp({4 * B.x - 3 * A.x, 4 * B.y - 3 * A.y});
                V2 dB = perp({3 * B.x - 4 * A.x, 3 * B.y - 4 * A.y});
                int eP = slot(ip, ip), eA = slot(ip, ia), eB = slot(ip, ib);
                P.sx[eP] -= (5.0 / 24.0) * dP.x; P.sy[eP] -= (5.0 / 24.0) * dP.y;
                P.sx[eA] -= dA.x / 24.0;         P.sy[eA] -= dA.y / 24.0;
                P.sx[eB] -= dB.x / 24.0;         P.sy[eB] -= dB.y / 24.0;
                P.cc[eP] += (11.0 / 54.0) * at;
                P.cc[eA] += (7.0 / 108.0) * at;
                P.cc[eB] += (7.0 / 108.0) * at;
                P.area[ip] += at / 3.0;
            }
    });
    // boundary edges (no reverse edge), then their half-edge fluxes in
    // (triangle, corner) order
    std::vector<uint8_t> bnd(3 * size_t(P.ntri), 0);
    parallel_for(P.ntri, [&](int t0, int t1) {
        for (int t = t0; t < t1; t++)
            for (int a = 0; a < 3; a++)
                bnd[3 * size_t(t) + a] = edge_far(P.tri[3 * t + (a + 1) % 3], P.tri[3 * t + a]) < 0;
    });
    for (int t = 0; t < P.ntri; t++)
        for (int a = 0; a < 3; a++) {
            int ia = P.tri[3 * t + a], ib = P.tri[3 * t + (a + 1) % 3];
            if (!bnd[3 * size_t(t) + a]) continue;  // interior edge
            V2 n = perp(sub(X(ib), X(ia)));
            int e;
            e = slot(ia, ia); P.sx[e] -= 0.375 * n.x; P.sy[e] -= 0.375 * n.y;
            e = slot(ia, ib); P.sx[e] -= 0.125 * n.x; P.sy[e] -= 0.125 * n.y;
            e = slot(ib, ib); P.sx[e] -= 0.375 * n.x; P.sy[e] -= 0.375 * n.y;
            e = slot(ib, ia); P.sx[e] -= 0.125 * n.x; P.sy[e] -= 0.125 * n.y;
        }
    parallel_for(P.n, [&](int p0, int p1) {
        for (int p = p0; p < p1; p++)
            for (int e = P.rowptr[p]; e < P.rowptr[p + 1]; e++) {
                P.sx[e] /= P.area[p];
                P.sy[e] /= P.area[p];
                P.cc[e] /= P.area[p];
            }
    });

    // ---- sub-steps: forward Euler stability of a mode damped at a = 1/tau_u
    // and oscillating at b = sqrt(2) max_P sum_k |s_Pk|: dt_u <= 2a/(a^2+b^2),
    // safety factor 1.1, at least the paper's n = 10
    if (o.n_sub > 0) {
        P.n_sub = o.n_sub;
    } else {
        std::vector<double> srow(P.n);
        parallel_for(P.n, [&](int p0, int p1) {
            for (int p = p0; p < p1; p++) {
                double s = 0.0;
                for (int e = P.rowptr[p]; e < P.rowptr[p + 1]; e++) s += std::hypot(P.sx[e], P.sy[e]);
                srow[p] = s;
            }
        });
        double smax = 0.0;
        for (int p = 0; p < P.n; p++) smax = std::max(smax, srow[p]);
        double a = 1.0 / P.tau_u, b = std::sqrt(2.0) * smax;
        double n = std::ceil(1.1 * (a * a + b * b) / (2.0 * a));
        P.n_sub = n < 10.0 ? 10 : int(n);
    }

    // ---- node order on the device: wall, fluid, ring; the fluid nodes follow a
    // Morton (Z-order) curve over their coordinates, so that a run of
    // consecutive rows is a compact patch of the mesh (the finite-volume kernel
    // stages each run's neighbourhood in shared memory)
    {
        double mx0 = 1e300, my0 = 1e300, mx1 = -1e300, my1 = -1e300;
        for (int p = 0; p < P.n; p++) {
            mx0 = std::min(mx0, P.xy[2 * p]); mx1 = std::max(mx1, P.xy[2 * p]);
            my0 = std::min(my0, P.xy[2 * p + 1]); my1 = std::max(my1, P.xy[2 * p + 1]);
        }
        double span = std::max(std::max(mx1 - mx0, my1 - my0), 1e-30);
        auto spread = [](uint32_t v) {  // 16 bits -> even bit positions
            uint64_t x = v & 0xffffu;
            x = (x | (x << 8)) & 0x00ff00ffu;
            x = (x | (x << 4)) & 0x0f0f0f0fu;
            x = (x | (x << 2)) & 0x33333333u;
            x = (x | (x << 1)) & 0x55555555u;
            return x;
        };
        std::vector<uint32_t> key(P.n);
        parallel_for(P.n, [&](int p0, int p1) {
            for (int p = p0; p < p1; p++) {
                uint32_t qx = uint32_t(std::min(65535.0, std::floor((P.xy[2 * p] - mx0) / span * 65535.0)));
                uint32_t qy = uint32_t(std::min(65535.0, std::floor((P.xy[2 * p + 1] - my0) / span * 65535.0)));
                key[p] = uint32_t(spread(qx) | (spread(qy) << 1));
            }
        });
        // wall and ring nodes keep their input order (the ring's interface data
        // and the wall edges are indexed in that order); fluid nodes are sorted
        // by key, equal keys in input order (a stable two-pass radix sort on
        // 16-bit digits of the 32-bit key)
        P.perm.clear();
        P.perm.reserve(P.n);
        for (int p = 0; p < P.n; p++)
            if (P.kind[p] == HLBM_NODE_WALL) P.perm.push_back(p);
        std::vector<int> fl, tmp;
        for (int p = 0; p < P.n; p++)
            if (P.kind[p] == HLBM_NODE_FLUID) fl.push_back(p);
        tmp.resize(fl.size());
        for (int shift : {0, 16}) {
            std::vector<int> cnt(65537, 0);
            for (int p : fl) cnt[((key[p] >> shift) & 0xffffu) + 1]++;
            for (int d = 0; d < 65536; d++) cnt[d + 1] += cnt[d];
            for (int p : fl) tmp[cnt[(key[p] >> shift) & 0xffffu]++] = p;
            fl.swap(tmp);
        }
        P.perm.insert(P.perm.end(), fl.begin(), fl.end());
        for (int p = 0; p < P.n; p++)
            if (P.kind[p] == HLBM_NODE_RING) P.perm.push_back(p);
    }
    P.inv.assign(P.n, 0);
    for (int q = 0; q < P.n; q++) P.inv[P.perm[q]] = q;
    P.n_wall = 0;
    P.n_ring = 0;
    for (int p = 0; p < P.n; p++) {
        P.n_wall += P.kind[p] == HLBM_NODE_WALL;
        P.n_ring += P.kind[p] == HLBM_NODE_RING;
    }
    P.ring_start = P.n - P.n_ring;
    for (int p = 0; p < P.n; p++)
        if (P.kind[p] == HLBM_NODE_RING) P.ring.push_back(p);

    // ---- wall edges: boundary edges between two wall nodes, in triangle order
    for (int t = 0; t < P.ntri; t++)
        for (int a = 0; a < 3; a++) {
            int ia = P.tri[3 * t + a], ib = P.tri[3 * t + (a + 1) % 3];
            if (P.kind[ia] != HLBM_NODE_WALL || P.kind[ib] != HLBM_NODE_WALL) continue;
            if (edge_far(ib, ia) >= 0) continue;
            P.wea.push_back(ia);
            P.web.push_back(ib);
        }

    // ---- wall nodes for the wall coefficients: N_P from the edge normals,
    // downstream tangent, body-frame chord position (pivot = quarter chord)
    {
        std::vector<double> N(2 * size_t(P.n), 0.0);
        for (size_t e = 0; e < P.wea.size(); e++) {
            const int a = P.wea[e], b = P.web[e];
            const double ex = P.xy[2 * b] - P.xy[2 * a], ey = P.xy[2 * b + 1] - P.xy[2 * a + 1];
            for (int v : {a, b}) {
                N[2 * v] -= 0.5 * ey;
                N[2 * v + 1] += 0.5 * ex;
            }
        }
        const double chx = ca, chy = -sa;  // chord direction after the rotation
        for (int p = 0; p < P.n; p++) {
            if (P.kind[p] != HLBM_NODE_WALL) continue;
            const double A = std::hypot(N[2 * p], N[2 * p + 1]);
            if (!(A > 0.0)) { err = "wall node without wall edges"; return HLBM_EINVAL; }
            const double nx = N[2 * p] / A, ny = N[2 * p + 1] / A;
            double sx = -ny, sy = nx;
            if (sx * chx + sy * chy < 0.0) { sx = -sx; sy = -sy; }
            const double bx = m->xy[2 * p] - px, by = m->xy[2 * p + 1] - py;  // input pose
            const double g7[7] = {bx / m->chord + 0.25, by >= 0.0 ? 1.0 : -1.0, A, nx, ny, sx, sy};
            P.wall_geo.insert(P.wall_geo.end(), g7, g7 + 7);
        }
    }

    // ---- finest level: nodes inside the rotated hole ellipse are not computed.
    // Membership: rotate the node back by +alpha about the pivot and test
    // ((X - cx)/a)^2 + ((Y - cy)/b)^2 < 1 (this arithmetic is fixed so that
    // every implementation classifies the same nodes).
    LevelPlan &F = P.lv[P.L - 1];
    const double *H = m->hole;
    if (!(H[2] > 0.0) || !(H[3] > 0.0)) { err = "hole semi-axes must be positive"; return HLBM_EINVAL; }
    std::vector<uint8_t> inhole(size_t(F.nx) * F.ny, 0);
    F.hx0.assign(F.ny, 0);
    F.hx1.assign(F.ny, 0);
    {
        // rows in parallel; the first failing row (in row order) names the error
        std::vector<uint8_t> row_err(F.ny, 0);  // 1: reaches a boundary, 2: not contiguous
        parallel_for(F.ny, [&](int y0, int y1) {
            for (int y = y0; y < y1; y++) {
                int first = -1, last = -2;
                for (int x = 0; x < F.nx && !row_err[y]; x++) {
                    double dx = double(x) - px, dy = double(y) - py;
                    double Xr = (ca * dx - sa * dy) + px - H[0];
                    double Yr = (sa * dx + ca * dy) + py - H[1];
                    double qx = Xr / H[2], qy = Yr / H[3];
                    if (qx * qx + qy * qy < 1.0) {
                        if (x == 0 || y == 0 || x == F.nx - 1 || y == F.ny - 1) { row_err[y] = 1; break; }
                        if (first < 0) first = x;
                        else if (x != last + 1) { row_err[y] = 2; break; }
                        last = x;
                        inhole[size_t(y) * F.nx + x] = 1;
                    }
                }
                if (!row_err[y] && first >= 0) { F.hx0[y] = first; F.hx1[y] = last + 1; }
            }
        }, 16);
        for (int y = 0; y < F.ny; y++) {
            if (row_err[y] == 1) { err = "hole reaches a level boundary"; return HLBM_EINVAL; }
            if (row_err[y] == 2) { err = "hole row is not contiguous"; return HLBM_EINVAL; }
        }
    }
    // coarser levels: a covered node whose coincident finer node is not computed
    // is not computed either (per row again one interval)
    for (int c = P.L - 2; c >= 0; c--) {
        LevelPlan &pa = P.lv[c];
        const LevelPlan &ch = P.lv[c + 1];
        pa.hx0.assign(pa.ny, 0);
        pa.hx1.assign(pa.ny, 0);
        for (int Y = pa.coy + 1; Y <= pa.coy + pa.cmy - 1; Y++) {
            int j = 2 * (Y - pa.coy);
            int a = ch.hx0[j], b = ch.hx1[j];
            if (a >= b) continue;
            int X0 = std::max(pa.cox + (a + 1) / 2, pa.cox + 1);
            int X1 = std::min(pa.cox + (b - 1) / 2, pa.cox + pa.cmx - 1);
            if (X0 <= X1) { pa.hx0[Y] = X0; pa.hx1[Y] = X1 + 1; }
        }
    }
    // structured interpolation nodes: hole nodes with a computed D2Q9 neighbour
    static const int ex[8] = {1, 0, -1, 0, 1, -1, -1, 1}, ey[8] = {0, 1, 0, -1, 1, 1, -1, -1};
    {
        std::vector<std::vector<int>> per_row(F.ny);
        parallel_for(F.ny - 2, [&](int j0, int j1) {
            for (int y = j0 + 1; y < j1 + 1; y++)
                for (int x = std::max(1, F.hx0[y]); x < std::min(F.nx - 1, F.hx1[y]); x++) {
                    if (!inhole[size_t(y) * F.nx + x]) continue;
                    bool near = false;
                    for (int d = 0; d < 8; d++) near |= !inhole[size_t(y + ey[d]) * F.nx + x + ex[d]];
                    if (near) per_row[y].push_back(y * F.nx + x);
                }
        }, 16);
        for (int y = 1; y < F.ny - 1; y++) P.is_node.insert(P.is_node.end(), per_row[y].begin(), per_row[y].end());
    }

    // ---- Eq. 8 stencils: containing triangle (lowest index when on an edge)
    // plus the far vertex across each of its three edges (Section 3, Fig. 1)
    double bx0 = 1e300, by0 = 1e300, bx1 = -1e300, by1 = -1e300;
    for (int p = 0; p < P.n; p++) {
        bx0 = std::min(bx0, P.xy[2 * p]); bx1 = std::max(bx1, P.xy[2 * p]);
        by0 = std::min(by0, P.xy[2 * p + 1]); by1 = std::max(by1, P.xy[2 * p + 1]);
    }
    const double cell = 2.0;
    int gw = int((bx1 - bx0) / cell) + 1, gh = int((by1 - by0) / cell) + 1;
    std::vector<std::vector<int>> bucket(size_t(gw) * gh);
    // only the buckets that hold an interpolation node are filled
    std::vector<uint8_t> need(size_t(gw) * gh, 0);
    int ni0 = gw, ni1 = -1, nj0 = gh, nj1 = -1;  // bucket range holding them
    for (int node : P.is_node) {
        double x = double(node % F.nx), y = double(node / F.nx);
        if (x >= bx0 && x <= bx1 && y >= by0 && y <= by1) {
            const int i = int((x - bx0) / cell), j = int((y - by0) / cell);
            need[size_t(j) * gw + i] = 1;
            ni0 = std::min(ni0, i); ni1 = std::max(ni1, i); nj0 = std::min(nj0, j); nj1 = std::max(nj1, j);
        }
    }
    {
        // triangle chunks in parallel, each listing (bucket, triangle) in
        // triangle order; appended chunk by chunk, so every bucket lists its
        // triangles in ascending order
        std::mutex part_mx;
        std::vector<std::pair<int, std::vector<std::pair<size_t, int>>>> parts;
        parallel_for(P.ntri, [&](int t0, int t1) {
            std::vector<std::pair<size_t, int>> mine;
            for (int t = t0; t < t1; t++) {
                double x0 = 1e300, y0 = 1e300, x1 = -1e300, y1 = -1e300;
                for (int a = 0; a < 3; a++) {
                    V2 q = X(P.tri[3 * t + a]);
                    x0 = std::min(x0, q.x); x1 = std::max(x1, q.x); y0 = std::min(y0, q.y); y1 = std::max(y1, q.y);
                }
                int i0 = int((x0 - bx0) / cell), i1 = int((x1 - bx0) / cell);
                int j0 = int((y0 - by0) / cell), j1 = int((y1 - by0) / cell);
                i0 = std::max(i0, ni0); i1 = std::min(i1, ni1); j0 = std::max(j0, nj0); j1 = std::min(j1, nj1);
                for (int j = j0; j <= j1; j++)
                    for (int i = i0; i <= i1; i++)
                        if (need[size_t(j) * gw + i]) mine.push_back({size_t(j) * gw + i, t});
            }
            std::lock_guard<std::mutex> lk(part_mx);
            parts.push_back({t0, std::move(mine)});
        });
        std::sort(parts.begin(), parts.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
        for (const auto &pt : parts)
            for (const auto &bt : pt.second) bucket[bt.first].push_back(bt.second);
    }
    const size_t nis = P.is_node.size();
    P.is_don.resize(6 * nis);
    P.is_w.resize(6 * nis);
    for (size_t s = 0; s < nis; s++) {
        double x = double(P.is_node[s] % F.nx), y = double(P.is_node[s] / F.nx);
        int found = -1;
        if (x >= bx0 && x <= bx1 && y >= by0 && y <= by1) {
            const std::vector<int> &cand = bucket[size_t(int((y - by0) / cell)) * gw + int((x - bx0) / cell)];
            for (int t : cand) {  // ascending triangle index
                V2 a = X(P.tri[3 * t]), b = X(P.tri[3 * t + 1]), c = X(P.tri[3 * t + 2]);
                double s0 = (b.x - x) * (c.y - y) - (b.y - y) * (c.x - x);
                double s1 = (c.x - x) * (a.y - y) - (c.y - y) * (a.x - x);
                double s2 = (a.x - x) * (b.y - y) - (a.y - y) * (b.x - x);
                if (s0 >= 0.0 && s1 >= 0.0 && s2 >= 0.0) { found = t; break; }
            }
        }
        if (found < 0) { err = "a structured interpolation node lies outside the mesh"; return HLBM_EINVAL; }
        int *d = &P.is_don[6 * s];
        for (int a = 0; a < 3; a++) d[a] = P.tri[3 * found + a];
        for (int a = 0; a < 3; a++) {
            int e0 = P.tri[3 * found + (a + 1) % 3], e1 = P.tri[3 * found + (a + 2) % 3];
            const int far = edge_far(e1, e0);
            if (far < 0) { err = "an interpolation triangle touches the mesh boundary"; return HLBM_EINVAL; }
            d[3 + a] = far;
        }
        // psi_k reproduce {1, X, Y, X^2, XY, Y^2} exactly at (x, y):
        // sum_k psi_k m_j(x_k - x) = m_j(0)
        double h = 0.0;
        for (int k = 0; k < 6; k++) {
            V2 q = X(d[k]);
            h = std::max(h, std::max(std::fabs(q.x - x), std::fabs(q.y - y)));
        }
        double A[36], rhs[6] = {1, 0, 0, 0, 0, 0};
        for (int k = 0; k < 6; k++) {
            V2 q = X(d[k]);
            double u = (q.x - x) / h, v = (q.y - y) / h;
            double mono[6] = {1.0, u, v, u * u, u * v, v * v};
            for (int j = 0; j < 6; j++) A[j * 6 + k] = mono[j];
        }
        if (!gauss_jordan(6, A, rhs)) { err = "singular 6-node interpolation stencil"; return HLBM_EINVAL; }
        for (int k = 0; k < 6; k++) P.is_w[6 * s + k] = rhs[k];
    }

    // ---- Eq. 9 stencils: 3x3 block of finest-level nodes centred on the node
    // nearest to the ring node, biquadratic Lagrange weights
    P.ring_don.resize(9 * size_t(P.n_ring));
    P.ring_w.resize(9 * size_t(P.n_ring));
    for (int r = 0; r < P.n_ring; r++) {
        V2 q = X(P.ring[r]);
        int X0 = int(std::floor(q.x + 0.5)), Y0 = int(std::floor(q.y + 0.5));
        double fx = q.x - X0, fy = q.y - Y0;
        double lx[3] = {0.5 * fx * (fx - 1.0), 1.0 - fx * fx, 0.5 * fx * (fx + 1.0)};
        double ly[3] = {0.5 * fy * (fy - 1.0), 1.0 - fy * fy, 0.5 * fy * (fy + 1.0)};
        for (int b = 0; b < 3; b++)
            for (int a = 0; a < 3; a++) {
                int xx = X0 + a - 1, yy = Y0 + b - 1;
                if (xx < 0 || yy < 0 || xx >= F.nx || yy >= F.ny) { err = "a ring donor lies outside the finest level"; return HLBM_EINVAL; }
                if (inhole[size_t(yy) * F.nx + xx]) { err = "a ring donor lies inside the hole"; return HLBM_EINVAL; }
                P.ring_don[9 * size_t(r) + 3 * b + a] = yy * F.nx + xx;
                P.ring_w[9 * size_t(r) + 3 * b + a] = lx[a] * ly[b];
            }
    }
    return HLBM_OK;
}

}  // namespace hlbm
