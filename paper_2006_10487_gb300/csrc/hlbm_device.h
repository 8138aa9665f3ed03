// Device-side state of one HLBM context and the kernel launchers
// (implemented in kernels.cu for float and double storage).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace hlbm {

// One Cartesian level in the in-place (AA) layout: nine planes of
// (ny + 2) x pitch values (one halo node on each side), plane stride `stride`;
// node (x, y) sits at index (y + 1) * pitch + x + 1.  Values are deviations
// f_i - w_i.  With parity 0 the state of node n is plane i at n; with parity 1
// it is plane opp(i) at n - c_i.
struct DevLevel {
    int nx = 0, ny = 0, pitch = 0;
    size_t stride = 0;
    void *f = nullptr;
    int parity = 0;
    double tau = 0;
    int *hx0 = nullptr, *hx1 = nullptr;  // finest level: hole interval per row
    bool has_child = false;
    int cox = 0, coy = 0, cmx = 0, cmy = 0, band_n = 0;
    // [12][band_n] (rho, ux, uy, f^neq) of the band before (A) and after (B)
    // this level's step: two buffers whose roles swap every step of the level
    // (B of one step is A of the next: the restriction in between writes only
    // the child's strict interior, never the band)
    void *snapA = nullptr, *snapB = nullptr;
    void *snap[2] = {nullptr, nullptr};
    int spar = 0;  // snapA = snap[spar], snapB = snap[spar ^ 1]
};

// One tiling of the finite-volume sub-step kernel: tiles of `rows`
// consecutive device rows (= threads per block); tile t's staged list
// halo_nodes[halo_ptr[t] .. halo_ptr[t+1]) is its own rows, then the other
// nodes its rows touch (sorted); the operator entries (sliced ELL, see
// DevMesh) carry positions in that list, in an order chosen per slice for
// the shared-memory banks.
struct FvTiles {
    int rows = 0;  // 0: not built
    int n_tiles = 0, max_tile_ent = 0, max_halo = 0;
    void *ent = nullptr;
    int *halo_ptr = nullptr, *halo_nodes = nullptr;
    int pf_ahead[3] = {0, 0, 0};  // per register bound: resident blocks (tile distance of the L2 prefetch)
    size_t smem_bytes = 0;
};

// The triangular mesh in device order (wall nodes, fluid nodes, ring nodes).
struct DevMesh {
    int n = 0, Np = 0, n_wall = 0, ring_start = 0, n_ring = 0;
    void *g[2] = {nullptr, nullptr};  // [9][Np] (rho - 1, ux, uy, f^neq_3..8), double-buffered
    int gcur = 0;
    // Eq. 3 operators, sliced ELL with 32-row slices: entry e of row r sits at
    // slice_ptr[r / 32] + 32 e + r % 32 of the tiling's entries, as
    // (dt s_x, dt s_y, dt / tau_u C, column); slice_ptr has n_slices + 1
    // elements, and the rows / 32 slices of tile t are the contiguous block
    // [slice_ptr[(rows / 32) t], slice_ptr[(rows / 32) (t + 1)]) of at most
    // max_tile_ent entries
    int n_slices = 0;
    int *slice_ptr = nullptr, *slice_len = nullptr;
    // the tiling in use (kTileRows or kTileRowsWide rows) and, until the
    // autotuner has chosen, the other one
    FvTiles tl, tl_alt;
    // FP32 sub-step kernel bounded for 1, 3: 7 (wide tiles: 3); 2, 4: 8 (4)
    // blocks per SM; 3, 4 with the L2 prefetch of a later tile
    int fv_variant = 1;
    // [12][n_ring] Eq. 9 data at t and t + 1: two buffers whose roles swap
    // every finest step (the data at t + 1 of one step is the data at t of the
    // next: nothing writes the finest level's lattice in between)
    void *Q0 = nullptr, *Q1 = nullptr;
    void *Qb[2] = {nullptr, nullptr};
    int qpar = 0;  // Q0 = Qb[qpar], Q1 = Qb[qpar ^ 1]
    int n_is = 0;
    int *is_n = nullptr;    // padded finest-level index of each structured interpolation node
    int *is_don = nullptr;  // [n_is][6] device-order mesh nodes
    void *is_w = nullptr;   // [n_is][6]
    int *ring_don = nullptr;  // [n_ring][9] padded finest-level indices
    void *ring_w = nullptr;   // [n_ring][9]
    int n_edges = 0;
    int *wea = nullptr, *web = nullptr;  // wall edges, device-order nodes
    double *wn = nullptr;                // [n_edges][2] normal times length, into the fluid
    // wall coefficients (Eq. 12-13): per wall row, unit normal and downstream
    // tangent [n_wall][4]; FP64 sums of C_p, C_f, C_n [3][n_wall]
    int wall_stats = 0;
    double *wall_ns = nullptr, *wall_acc = nullptr;
    int *inv = nullptr;                  // input node -> device node
    void *lap = nullptr;                 // [9][Np] scratch of the odd-even filter (allocated when it is on)
};

// FP16S lattice storage shift: s_i = f^eq_i(1, (u0, 0)) - w_i (free stream).
struct LatShift {
    float s[9];
};

struct DevCtx {
    int L = 0;
    LatShift shift = {};
    DevLevel lv[8];
    DevMesh m;
    double u0 = 0, tau_u = 0, dt_u = 0, qdyn = 0;
    int n_sub = 0;
    double fv_filter = 0;  // odd-even filter strength per finest step (0: off)
    double *force_buf = nullptr;  // [force_cap][2]
    double *force_partial = nullptr;  // [ceil(n_edges / 128)][2] per-block partial sums
    int *force_counter = nullptr;
    int *flag = nullptr;
    int force_cap = 0;
};

constexpr int kTileRows = 128;       // rows per finite-volume tile (= threads per block)
constexpr int kTileRowsWide = 256;   // the wide tiling the FP32 autotuner also times

// Launchers, T = arithmetic type, S = lattice storage type (T, or __half for
// FP16S); raises the FV kernel's dynamic shared-memory limit (configure_fv).
template <typename T, typename S> void configure_fv(const FvTiles &tl);
// resident blocks of each sub-step kernel variant of a tiling (tl.pf_ahead)
template <typename T, typename S> void configure_fv_prefetch(FvTiles &tl);
// times the FP32 sub-step kernel's four variants on this mesh's tiling
// (us[0..3]) and on the wide tiling if built (us[4..7]); leaves the fastest
// in m.tl / m.fv_variant (the other tiling in m.tl_alt, for the caller to
// free) and returns it as 1..4 (tiles of kTileRows) or 5..8 (wide tiles)
template <typename T, typename S> int fv_autotune(DevCtx &, cudaStream_t, double us[8]);
template <typename T, typename S> void launch_init_level(const DevCtx &, int c, unsigned long long seed, double perturb, cudaStream_t);
template <typename T, typename S> void launch_collide(const DevCtx &, int c, cudaStream_t);
template <typename T, typename S> void launch_outer_bc(const DevCtx &, cudaStream_t);
template <typename T, typename S> void launch_snapshot(const DevCtx &, int c, bool into_b, cudaStream_t);
template <typename T, typename S> void launch_prolong(const DevCtx &, int c_fine, double theta, cudaStream_t);
template <typename T, typename S> void launch_restrict(const DevCtx &, int c_coarse, cudaStream_t);
template <typename T, typename S> void launch_ring_interp(const DevCtx &, bool q1_and_star, cudaStream_t);
template <typename T, typename S> void launch_hole_interp(const DevCtx &, cudaStream_t);
template <typename T, typename S> void launch_fv(const DevCtx &, int m, cudaStream_t);
// FP32 -> FP64 copy of n values
void launch_widen(const float *a, double *b, size_t n, cudaStream_t);
// odd-even filter of the mesh state (g[gcur] -> g[gcur ^ 1]); no launch when off
template <typename T, typename S> void launch_fv_filter(const DevCtx &, cudaStream_t);
template <typename T, typename S> void launch_forces(const DevCtx &, cudaStream_t);
// FP64 total of sum_i (f_i - w_i) over level 0's computed nodes into out[0] (row_sum: ny0 doubles)
template <typename T, typename S> void launch_mass(const DevCtx &, double *row_sum, double *out, cudaStream_t);
// adds this state's wall coefficients to the sums (Eq. 12-13)
template <typename T, typename S> void launch_wall_stats(const DevCtx &, cudaStream_t);
template <typename T, typename S> void launch_fields(const DevCtx &, int grid, double *rho, double *ux, double *uy, double *pop, cudaStream_t);
// Device tables of the finite-volume adjoint (FP64), device node order.
struct AdjTables {
    bool built = false;
    // off-diagonal Eq. 3 entries of each row: columns, (dt s_x, dt s_y,
    // dt / tau_u C), index of the entry in the plan's CSR
    int *rp = nullptr, *rcol = nullptr, *rcsr = nullptr;
    double *rcoef = nullptr;
    // rows reading node Q: trow[tp[Q] .. tp[Q + 1]), with the position of Q
    // in that row's entries (-1: the row of Q itself)
    int *tp = nullptr, *trow = nullptr, *tpos = nullptr;
    // wall edges (device-order end nodes, normal times length) and the edges
    // of each node: wedge[wptr[Q] .. wptr[Q + 1])
    int n_edges = 0;
    int *wea = nullptr, *web = nullptr, *wptr = nullptr, *wedge = nullptr;
    double *wn = nullptr;
    int *perm = nullptr;  // device node -> input node
    // geometry (input node order) for dJ / d(node coordinates): the plan's CSR
    // operators (s_x, s_y, C) and control-volume areas, posed coordinates,
    // triangles and the triangles of each node, boundary edges (a -> b, no
    // reverse edge) and wall edges of each node
    int n_tri = 0, n_bedge = 0;
    int *prow = nullptr, *pcol = nullptr, *ptri = nullptr, *ntp = nullptr, *ntl = nullptr;
    double *pcoef = nullptr, *parea = nullptr, *pxy = nullptr;
    int *bed = nullptr, *bptr = nullptr, *blist = nullptr;
    int *iwea = nullptr, *iweb = nullptr, *iwptr = nullptr, *iwlist = nullptr;
    int *inv = nullptr;  // input node -> device node
    // coupled step (single level): the (ring node, donor) pairs of Eq. 9 per
    // finest-level node, lent[lptr[y nx + x] ..) as 9 r + k, and the
    // (interpolation node, donor) pairs of Eq. 8 per device mesh node,
    // hent[hptr[node] ..) as 6 s + k
    int *lptr = nullptr, *lent = nullptr, *hptr = nullptr, *hent = nullptr;
    // prolongation into level l: the (fine perimeter node, weight) pairs of
    // each band entry of level l - 1, pk[l][pp[l][b] ..), weights pw[l]
    int *pp[8] = {}, *pk[8] = {};
    double *pw[8] = {};
    // Eq. 8 stencils in input order: donors [n_is][6] and the interpolation
    // nodes' lattice coordinates [n_is][2] (finest units)
    int *isd_in = nullptr;
    double *is_xy = nullptr;
    bool coupled_built = false;
};
void launch_adj_value(const AdjTables &, const double *g, int Np, double wd, double wl, double inv_q, double *J,
                      cudaStream_t);
void launch_adj_terminal(const AdjTables &, const double *g, int Np, int n, double wd, double wl, double inv_q,
                         double *lam, cudaStream_t, bool add = false);
// scratch: 27 Np doubles (per-row mu, sig, E of the reverse sub-step)
void launch_fv_adjoint(const AdjTables &, const double *g, int Np, int n, double csP, int n_wall, int ring_start,
                       int star, double dt, double dt_tau, const double *lam_in, double *lam_out, double *gcoef,
                       double *scratch, cudaStream_t);
void launch_adj_populations(const AdjTables &, const double *g, int Np, int n, const double *lam, double *grad,
                            cudaStream_t);
// dJ/d(node coordinates) from the operator-entry gradient gc ([nnz][3], plan
// order) and the wall normals of the final state gM; grad_xy [n][2] in the
// input frame, dJ / d(angle of attack, per degree) into *daoa.  scratch:
// n + 2 n_wall_edges + 2 n doubles.
void launch_adj_geometry(const AdjTables &, int n, const double *gc, const double *gM, int Np, double wd, double wl,
                         double inv_q, double ca, double sa, double px, double py, double *scratch, double *grad_xy,
                         double *daoa, cudaStream_t);

// adjoints of the lattice side of a single-level coupled step (FP64, parity P)
void launch_adj_collide(const DevLevel &, const double *f, int P, double *lam, cudaStream_t);
void launch_adj_outer_bc(const DevLevel &, const double *f, int P, double u0, double *lam, cudaStream_t);
void launch_adj_ring_lattice(const DevLevel &, const double *f, int P, const AdjTables &, const double *ring_w,
                             const double *lamQ, int n_ring, double *lam, cudaStream_t);
// lamq: 12 n_is doubles of scratch
// lw6 (optional): dJ/d(Eq. 8 weights) [n_is][6], accumulated
void launch_adj_hole(const DevLevel &, const DevMesh &, const AdjTables &, const double *g, int P, double *lam,
                     double *lamq, double *lam_g, cudaStream_t, double *lw6 = nullptr);
void launch_adj_ring_rows(const DevMesh &, double scale5, double wa, double wb, double *lam_g, double *lamQ0,
                          double *lamQ1, cudaStream_t);
void launch_adj_lattice_out(const DevLevel &, const double *lam, int P, double *grad, cudaStream_t);
// geometry through the coupled step: Eq. 9 weight cotangents (accumulated),
// then dJ/dx (input frame) and dJ/d(angle of attack) from the accumulated
// entry, wall-normal (hacc [n_wall_edges][2]), Eq. 8 and Eq. 9 weight
// cotangents; scratch: 3 n + 6 n_is doubles
void launch_adj_ring_weights(const DevLevel &, const DevMesh &, const double *f, int P, const double *lamQ, double *lw9,
                             cudaStream_t);
void launch_adj_geometry_coupled(const AdjTables &, const DevMesh &, int n, const double *gc, const double *hacc,
                                 const double *lw6, const double *lw9, double ca, double sa, double px, double py,
                                 double *scratch, double *grad_xy, double *daoa, cudaStream_t);
void launch_adj_wall_normal(const AdjTables &, const double *g, int Np, double wd, double wl, double inv_q,
                            double *hacc, cudaStream_t);
// refinement interface: band snapshot of parent l, prolongation into l (lamq:
// 12 x perimeter(l) doubles of scratch), restriction into parent p from l
void launch_adj_snapshot(const DevLevel &, const double *f, int P, const double *lamS, double *lam, cudaStream_t);
void launch_adj_prolong(const DevLevel &parent, const DevLevel &l, int P, double theta, const double *A,
                        const double *B, const int *pp, const int *pk, const double *pw, double *lam, double *lamq,
                        double *lamA, double *lamB, cudaStream_t);
void launch_adj_restrict(const DevLevel &parent, const DevLevel &l, int PC, int PF, const double *ff, double *lamc,
                         double *lamf, cudaStream_t);

// bounds-checked build (HLBM_DEBUG): violations so far and the bit mask of the
// sites that saw them, for the whole process; returns false (out = 0) in a
// build without the checks
bool debug_bounds(unsigned int out[2]);

}  // namespace hlbm
