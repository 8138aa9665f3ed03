/*
 * HLBM oracle: a plain, slow, double-precision CPU implementation of the
 * hybrid lattice Boltzmann method (Di Ilio, Chiappini, Ubertini, Bella, Succi,
 * "Fluid flow around NACA 0012 airfoil at low-Reynolds numbers with hybrid
 * lattice Boltzmann method").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker for the CUDA library; it
 * shares no code, header, table or helper with it.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Layout: every grid is stored node-major (the nine populations of a node are
 * contiguous) and double-buffered; streaming is a plain pull from the
 * upstream node.  Each step of the method is one straightforward loop.
 *
 * Paper passages followed:
 *   Eq. 1  structured BGK lattice Boltzmann equation (Section 2)
 *   Eq. 2  equilibrium distribution (Section 2)
 *   Eq. 3  cell-vertex finite-volume LBE on the triangular mesh (Section 2)
 *   Eq. 4  post-collision state of structured interpolation nodes (Section 2)
 *   Eq. 5-7 post-collision state of unstructured interpolation nodes (Section 2)
 *   Eq. 8  6-node quadratic interpolation, triangles -> lattice (Section 3)
 *   Eq. 9  9-node quadratic interpolation, lattice -> triangles (Section 3)
 *   Section 4: nested factor-2 refinement boxes, wall and outer conditions
 *   Eq. 10-11 drag and lift coefficients (Section 6.1)
 * Where the paper leaves a step unspecified the reading used here is stated
 * at the function that implements it.
 *
 * Built with -fopenmp, the loops over independent nodes run on several host
 * threads; every output value is written by one iteration from inputs no
 * iteration writes, in the same order of operations, so the results are
 * bitwise those of the serial build.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- D2Q9 ---- */
/* Velocity set and weights: the standard D2Q9 choice (the paper names D2Q9-type
 * weights normalised to one and the lattice sound speed, c_s^2 = 1/3). */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WQ[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* Eq. 2 with c_s^2 = 1/3:
 * f_i^eq = w_i rho [1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u]. */
void orc_feq(double rho, double ux, double uy, double *out)
{
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; i++) {
        double cu = CX[i] * ux + CY[i] * uy;
        out[i] = WQ[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* Zeroth and first moments: rho = sum f, rho u = sum c f. */
void orc_moments(const double *f, double *rho, double *ux, double *uy)
{
    double r = 0.0, mx = 0.0, my = 0.0;
    for (int i = 0; i < 9; i++) {
        r += f[i];
        mx += CX[i] * f[i];
        my += CY[i] * f[i];
    }
    *rho = r;
    *ux = mx / r;
    *uy = my / r;
}

/* Macroscopic state plus non-equilibrium part: q = (rho, ux, uy, f - f^eq). */
static void state_q(const double *f, double *q)
{
    double eq[9];
    orc_moments(f, &q[0], &q[1], &q[2]);
    orc_feq(q[0], q[1], q[2], eq);
    for (int i = 0; i < 9; i++) q[3 + i] = f[i] - eq[i];
}

/* f^neq has zero mass and momentum by definition (f^eq shares rho and rho u
 * with f): sum_i f^neq_i = 0, sum_i c_i f^neq_i = 0.  Enforce it on a stored
 * state q = (rho, u, f^neq) by solving the three relations for f^neq_0..2:
 *   f^neq_1 = f^neq_3 - f^neq_5 + f^neq_6 + f^neq_7 - f^neq_8
 *   f^neq_2 = f^neq_4 - f^neq_5 - f^neq_6 + f^neq_7 + f^neq_8
 *   f^neq_0 = -(f^neq_1 + ... + f^neq_8)
 * (otherwise rounding lets the constraints drift, and the collision term of
 * Eq. 3 turns the drift into spurious mass and momentum sources). */
static void neq_constrain(double *q)
{
    double *n = q + 3;
    n[1] = n[3] - n[5] + n[6] + n[7] - n[8];
    n[2] = n[4] - n[5] - n[6] + n[7] + n[8];
    n[0] = -(n[1] + n[2] + n[3] + n[4] + n[5] + n[6] + n[7] + n[8]);
}

/* Population from (rho, u, f^neq) with the non-equilibrium part scaled:
 * f = f^eq(rho, u) + scale * f^neq. */
static void from_q(const double *q, double scale, double *f)
{
    double eq[9];
    orc_feq(q[0], q[1], q[2], eq);
    for (int i = 0; i < 9; i++) f[i] = eq[i] + scale * q[3 + i];
}

/* f^eq_i(rho_a, u_a) - f^eq_i(rho_b, u_b) written through the differences of
 * the moments (Eq. 2):  w_i [ (rho_a - rho_b) E_i(u_b) + rho_a (E_i(u_a) - E_i(u_b)) ]
 * with E_i(u) = 1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u and
 * E_i(u_a) - E_i(u_b) = 3 c.du + 9/2 (c.du)(c.(u_a + u_b)) - 3/2 du.(u_a + u_b),
 * du = u_a - u_b; no large terms cancel. */
void orc_feq_diff(double ra, double uax, double uay, double rb, double ubx, double uby, double *out)
{
    double dux = uax - ubx, duy = uay - uby, sux = uax + ubx, suy = uay + uby;
    double ub2 = ubx * ubx + uby * uby, dus = dux * sux + duy * suy;
    for (int i = 0; i < 9; i++) {
        double cub = CX[i] * ubx + CY[i] * uby;
        double cdu = CX[i] * dux + CY[i] * duy, csu = CX[i] * sux + CY[i] * suy;
        double eb = 1.0 + 3.0 * cub + 4.5 * cub * cub - 1.5 * ub2;
        double de = 3.0 * cdu + 4.5 * cdu * csu - 1.5 * dus;
        out[i] = WQ[i] * ((ra - rb) * eb + ra * de);
    }
}

/* Eq. 4: post-collision state of a structured interpolation node from
 * interpolated unstructured data q = (rho, u, f^neq,u):
 * f~s = f^eq + 2 (tau_s - 1) / (2 tau_s - 1) f^neq,u  (unit structured step). */
void orc_eq4_post(const double *q, double tau_s, double *f)
{
    from_q(q, 2.0 * (tau_s - 1.0) / (2.0 * tau_s - 1.0), f);
}

/* Eq. 5-6: the structured part of the state of an unstructured interpolation
 * node from interpolated lattice data q = (rho, u, f^neq,s): the same rho and
 * u with f^neq,u = (1 - 1/(2 tau_s)) f^neq,s (mesh state kept as (rho, u, f^neq)). */
static void eq5_q(const double *q, double tau_s, double *qu)
{
    qu[0] = q[0]; qu[1] = q[1]; qu[2] = q[2];
    for (int i = 0; i < 9; i++) qu[3 + i] = (1.0 - 1.0 / (2.0 * tau_s)) * q[3 + i];
    neq_constrain(qu);
}

/* The same as populations: f^eq,s + (1 - 1/(2 tau_s)) f^neq,s. */
void orc_eq5_base(const double *q, double tau_s, double *g)
{
    double qu[12];
    eq5_q(q, tau_s, qu);
    from_q(qu, 1.0, g);
}

/* Eq. 1 collision (right-hand side), unit time step on the grid's own clock:
 * f* = f - (f - f^eq) / tau. */
void orc_bgk_collide(double *f, double tau)
{
    double rho, ux, uy, eq[9];
    orc_moments(f, &rho, &ux, &uy);
    orc_feq(rho, ux, uy, eq);
    for (int i = 0; i < 9; i++) f[i] = f[i] - (f[i] - eq[i]) / tau;
}

/* Eq. 1 streaming by pulling from the upstream node:
 * f_i(x, t + 1) = f*_i(x - c_i, t).  Without wrap-around, a population whose
 * upstream node lies outside the grid is left undefined (NaN); the boundary
 * rules refill those nodes. */
static void stream_pull(const double *post, double *f, int nx, int ny, int periodic)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++)
            for (int i = 0; i < 9; i++) {
                int xs = x - CX[i], ys = y - CY[i];
                double v = NAN;
                if (periodic) { xs = (xs + nx) % nx; ys = (ys + ny) % ny; }
                if (xs >= 0 && xs < nx && ys >= 0 && ys < ny) v = post[9 * ((size_t)ys * nx + xs) + i];
                f[9 * ((size_t)y * nx + x) + i] = v;
            }
}

/* Eq. 1 on a fully periodic nx x ny lattice: collide, then stream.
 * Used by the lattice pins. */
void orc_lattice_periodic(double *f, int nx, int ny, double tau, int nsteps)
{
    size_t n = (size_t)nx * ny;
    double *post = malloc(n * 9 * sizeof(double));
    for (int s = 0; s < nsteps; s++) {
        memcpy(post, f, n * 9 * sizeof(double));
        for (size_t p = 0; p < n; p++) orc_bgk_collide(post + 9 * p, tau);
        stream_pull(post, f, nx, ny, 1);
    }
    free(post);
}

/* ------------------------------------------------- random initial state --- */
/* splitmix64 (Steele, Lea, Flood 2014), one output from state s. */
static uint64_t splitmix64(uint64_t s)
{
    uint64_t z = s + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Uniform deviate in [-1, 1) for node `idx` of grid `gid`. */
double orc_uniform(uint64_t seed, uint64_t gid, uint64_t idx)
{
    uint64_t z = splitmix64(seed ^ (gid << 40) ^ idx);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

/* ------------------------------------------------------- edge table ----- */
/* Directed edges (a -> b) of counter-clockwise triangles, sorted by key, so
 * that the triangle across an edge is found by looking up (b -> a). */
typedef struct { uint64_t key; int tri, far; } oedge;

static int edge_cmp(const void *x, const void *y)
{
    uint64_t a = ((const oedge *)x)->key, b = ((const oedge *)y)->key;
    return a < b ? -1 : (a > b ? 1 : 0);
}

static oedge *edge_table(int ntri, const int *tri)
{
    oedge *e = malloc((size_t)(3 * ntri > 0 ? 3 * ntri : 1) * sizeof(oedge));
    for (int t = 0; t < ntri; t++)
        for (int a = 0; a < 3; a++) {
            oedge *d = &e[3 * t + a];
            d->key = ((uint64_t)(uint32_t)tri[3 * t + a] << 32) | (uint32_t)tri[3 * t + (a + 1) % 3];
            d->tri = t;
            d->far = tri[3 * t + (a + 2) % 3];
        }
    qsort(e, (size_t)3 * ntri, sizeof(oedge), edge_cmp);
    return e;
}

/* The entry of directed edge (a -> b), or NULL when no triangle holds it. */
static const oedge *edge_find(const oedge *e, int ntri, int a, int b)
{
    oedge k;
    k.key = ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
    return bsearch(&k, e, (size_t)3 * ntri, sizeof(oedge), edge_cmp);
}

/* ------------------------------------------- finite-volume operators ------ */
/* Eq. 3 coefficients.  The paper omits their derivation; the reading used is
 * the cell-vertex (median-dual) finite volume with a piecewise-linear field in
 * every triangle.  The control volume of node P is the union, over triangles
 * T = (P, A, B) around P, of the quadrilateral (P, M_PA, G_T, M_PB), where M
 * are edge midpoints and G_T the centroid; its area is A_P = sum A_T / 3.
 *
 * Streaming: -(1/A_P) * contour integral of (c_i . n) f, integrated exactly for
 * the linear field (segment length times the value at its midpoint):
 *   segment M_PA -> G_T has midpoint weights (P, A, B) = (5/12, 5/12, 1/6),
 *   segment G_T -> M_PB has (5/12, 1/6, 5/12),
 *   a boundary half edge P -> M_PA (edge PA on the mesh boundary) has (3/4, 1/4, 0).
 * Hence S_ik = c_i . s_k with s_k = -(1/A_P) sum_seg (n L)_seg w_seg,k.
 *
 * Collision: C_Pk = (1/A_P) * integral over the control volume of the hat
 * function of node k: 11/54 A_T per triangle for k = P and 7/108 A_T per
 * triangle holding edge Pk.
 *
 * tri_xy (optional, [ntri][3][2]) gives per-triangle vertex coordinates, so a
 * periodic mesh can pass unwrapped coordinates; NULL means xy[tri].
 * Row P of the output holds P and its edge neighbours, sorted by column.
 * Output arrays need room for n + 6*ntri entries.  Returns nnz, or -1 on an
 * inverted or degenerate triangle. */
int orc_fv_operators(int n, const double *xy, int ntri, const int *tri, const double *tri_xy,
                     int *rowptr, int *col, double *sx, double *sy, double *cc, double *area)
{
    /* neighbour lists: candidate columns per row, deduplicated below */
    int cap = n + 6 * ntri;
    int *deg = calloc((size_t)n + 1, sizeof(int));
    for (int t = 0; t < ntri; t++)
        for (int a = 0; a < 3; a++) deg[tri[3 * t + a]] += 2;
    int *start = malloc(((size_t)n + 1) * sizeof(int));
    start[0] = 0;
    for (int p = 0; p < n; p++) start[p + 1] = start[p] + deg[p] + 1;
    int *cand = malloc((size_t)start[n] * sizeof(int));
    int *fill = calloc((size_t)n, sizeof(int));
    for (int p = 0; p < n; p++) cand[start[p] + fill[p]++] = p;
    for (int t = 0; t < ntri; t++)
        for (int a = 0; a < 3; a++) {
            int p = tri[3 * t + a];
            cand[start[p] + fill[p]++] = tri[3 * t + (a + 1) % 3];
            cand[start[p] + fill[p]++] = tri[3 * t + (a + 2) % 3];
        }
    /* sort + unique each candidate list (insertion sort; lists are short) */
    int nnz = 0;
    rowptr[0] = 0;
    for (int p = 0; p < n; p++) {
        int *c = cand + start[p];
        int m = fill[p];
        for (int i = 1; i < m; i++) {
            int v = c[i], j = i - 1;
            while (j >= 0 && c[j] > v) { c[j + 1] = c[j]; j--; }
            c[j + 1] = v;
        }
        for (int i = 0; i < m; i++)
            if (i == 0 || c[i] != c[i - 1]) {
                if (nnz >= cap) { nnz = -1; goto done; }
                col[nnz] = c[i];
                sx[nnz] = sy[nnz] = cc[nnz] = 0.0;
                nnz++;
            }
        rowptr[p + 1] = nnz;
    }
    for (int p = 0; p < n; p++) area[p] = 0.0;

    /* boundary edges: an edge used by exactly one triangle */
    /* count uses of directed edge (a,b) by looking up (b,a) */
    for (int t = 0; t < ntri; t++) {
        double v[3][2];
        for (int a = 0; a < 3; a++) {
            if (tri_xy) { v[a][0] = tri_xy[6 * t + 2 * a]; v[a][1] = tri_xy[6 * t + 2 * a + 1]; }
            else { v[a][0] = xy[2 * tri[3 * t + a]]; v[a][1] = xy[2 * tri[3 * t + a] + 1]; }
        }
        double at = 0.5 * ((v[1][0] - v[0][0]) * (v[2][1] - v[0][1])
                           - (v[1][1] - v[0][1]) * (v[2][0] - v[0][0]));
        if (!(at > 0.0)) { nnz = -1; goto done; }
        for (int a = 0; a < 3; a++) {
            int ip = tri[3 * t + a], ia = tri[3 * t + (a + 1) % 3], ib = tri[3 * t + (a + 2) % 3];
            /* coordinates relative to P (P at the origin), so that the short
             * dual segments are not formed by cancelling large absolute
             * coordinates */
            double A[2] = {v[(a + 1) % 3][0] - v[a][0], v[(a + 1) % 3][1] - v[a][1]};
            double B[2] = {v[(a + 2) % 3][0] - v[a][0], v[(a + 2) % 3][1] - v[a][1]};
            double g[2] = {(A[0] + B[0]) / 3.0, (A[1] + B[1]) / 3.0};
            double mpa[2] = {0.5 * A[0], 0.5 * A[1]};
            double mpb[2] = {0.5 * B[0], 0.5 * B[1]};
            /* the sub-quad P, M_PA, G, M_PB is counter-clockwise, so the outward
             * normal times length of a directed edge (u -> v) is (dy, -dx) */
            double n1[2] = {g[1] - mpa[1], -(g[0] - mpa[0])};
            double n2[2] = {mpb[1] - g[1], -(mpb[0] - g[0])};
            /* accumulate -(n L) w into the row of P (divided by A_P afterwards) */
            int cols[3] = {ip, ia, ib};
            double w1[3] = {5.0 / 12.0, 5.0 / 12.0, 1.0 / 6.0};
            double w2[3] = {5.0 / 12.0, 1.0 / 6.0, 5.0 / 12.0};
            for (int k = 0; k < 3; k++) {
                int e;
                for (e = rowptr[ip]; e < rowptr[ip + 1]; e++)
                    if (col[e] == cols[k]) break;
                sx[e] -= n1[0] * w1[k] + n2[0] * w2[k];
                sy[e] -= n1[1] * w1[k] + n2[1] * w2[k];
                cc[e] += (k == 0 ? 11.0 / 54.0 : 7.0 / 108.0) * at;
            }
            area[ip] += at / 3.0;
        }
    }
    /* boundary half edges: edge (a,b) of triangle t is on the boundary when no
     * other triangle holds the reversed edge (b,a). */
    oedge *et = edge_table(ntri, tri);
    for (int t = 0; t < ntri; t++) {
        for (int a = 0; a < 3; a++) {
            int ia = tri[3 * t + a], ib = tri[3 * t + (a + 1) % 3];
            if (edge_find(et, ntri, ib, ia)) continue;
            double va[2], vb[2];
            if (tri_xy) {
                va[0] = tri_xy[6 * t + 2 * a]; va[1] = tri_xy[6 * t + 2 * a + 1];
                vb[0] = tri_xy[6 * t + 2 * ((a + 1) % 3)]; vb[1] = tri_xy[6 * t + 2 * ((a + 1) % 3) + 1];
            } else {
                va[0] = xy[2 * ia]; va[1] = xy[2 * ia + 1];
                vb[0] = xy[2 * ib]; vb[1] = xy[2 * ib + 1];
            }
            /* directed boundary edge a -> b (fluid on its left); outward n L = (dy, -dx).
             * Half edge a -> M_ab belongs to the control volume of a,
             * half edge M_ab -> b to that of b; each has half the edge's n L. */
            double nl[2] = {0.5 * (vb[1] - va[1]), -0.5 * (vb[0] - va[0])};
            int own[2] = {ia, ib}, oth[2] = {ib, ia};
            for (int s = 0; s < 2; s++) {
                int p = own[s];
                for (int e = rowptr[p]; e < rowptr[p + 1]; e++) {
                    if (col[e] == p) { sx[e] -= nl[0] * 0.75; sy[e] -= nl[1] * 0.75; }
                    if (col[e] == oth[s]) { sx[e] -= nl[0] * 0.25; sy[e] -= nl[1] * 0.25; }
                }
            }
        }
    }
    free(et);
    for (int p = 0; p < n; p++)
        for (int e = rowptr[p]; e < rowptr[p + 1]; e++) {
            sx[e] /= area[p];
            sy[e] /= area[p];
            cc[e] /= area[p];
        }
done:
    free(deg); free(start); free(cand); free(fill);
    return nnz;
}

/* Eq. 3, one explicit sub-step on every node (no wall or interface rule):
 * g'_i(P) = g_i(P) + dt sum_k S_ik g_i(P_k) - (dt/tau_u) sum_k C_Pk g^neq_i(P_k).
 * The mesh state is kept per node as q = (rho, ux, uy, g^neq_0..8), the
 * decomposition g = f^eq(rho, u) + g^neq of Eq. 4-7, so that g^neq is held
 * directly rather than recovered by cancelling two O(w_i) numbers.  The
 * control volume is closed (sum_k S_ik = 0), so the streaming sum is taken as
 * sum_k S_ik [g_i(P_k) - g_i(P)] with g(P_k) - g(P) = [f^eq(P_k) - f^eq(P)]
 * + [g^neq(P_k) - g^neq(P)] (orc_feq_diff).  The new state follows from
 * g' = g + acc: rho' = rho + sum acc, u' from the momentum, and
 * g^neq' = g^neq + acc - [f^eq(rho', u') - f^eq(rho, u)]. */
static void fv_substep_q(int n, const int *rowptr, const int *col, const double *sx, const double *sy,
                         const double *cc, double dt, double tau_u, const double *q, double *qn)
{
#pragma omp parallel for schedule(static)
    for (int p = 0; p < n; p++) {
        const double *qp = q + 12 * (size_t)p;
        double acc[9] = {0};
        for (int e = rowptr[p]; e < rowptr[p + 1]; e++) {
            const double *qk = q + 12 * (size_t)col[e];
            double dfe[9];
            orc_feq_diff(qk[0], qk[1], qk[2], qp[0], qp[1], qp[2], dfe);
            for (int i = 0; i < 9; i++) {
                double s = CX[i] * sx[e] + CY[i] * sy[e];
                acc[i] += dt * s * (dfe[i] + qk[3 + i] - qp[3 + i]) - (dt / tau_u) * cc[e] * qk[3 + i];
            }
        }
        double drho = 0.0, djx = 0.0, djy = 0.0;
        for (int i = 0; i < 9; i++) {
            drho += acc[i];
            djx += CX[i] * acc[i];
            djy += CY[i] * acc[i];
        }
        double *qo = qn + 12 * (size_t)p;
        double rho = qp[0] + drho;
        qo[0] = rho;
        qo[1] = qp[1] + (djx - drho * qp[1]) / rho;
        qo[2] = qp[2] + (djy - drho * qp[2]) / rho;
        double dfe[9];
        orc_feq_diff(qo[0], qo[1], qo[2], qp[0], qp[1], qp[2], dfe);
        for (int i = 0; i < 9; i++) qo[3 + i] = qp[3 + i] + acc[i] - dfe[i];
        neq_constrain(qo);
    }
}

/* Eq. 3 on populations g[n][9] (converted to and from the (rho, u, g^neq)
 * state around fv_substep_q). */
void orc_fv_substep(int n, const int *rowptr, const int *col, const double *sx, const double *sy,
                    const double *cc, double dt, double tau_u, const double *g, double *gnew)
{
    double *q = calloc((size_t)n * 12 + 1, sizeof(double)), *qn = calloc((size_t)n * 12 + 1, sizeof(double));
    for (int p = 0; p < n; p++) state_q(g + 9 * (size_t)p, q + 12 * (size_t)p);
    fv_substep_q(n, rowptr, col, sx, sy, cc, dt, tau_u, q, qn);
    for (int p = 0; p < n; p++) from_q(qn + 12 * (size_t)p, 1.0, gnew + 9 * (size_t)p);
    free(q);
    free(qn);
}

/* Eq. 3 exactly as printed, on populations g[n][9]:
 *   g'_i(P) = g_i(P) + dt sum_k S_ik g_i(P_k) - (dt/tau_u) sum_k C_ik [g_i(P_k) - f_i^eq(P_k)],
 * the sums running over P itself (k = 0) and its edge neighbours, with
 * S_ik = c_i . (s_x, s_y)_k and f^eq(P_k) of Eq. 2 from the moments of
 * g(P_k).  No (rho, u, g^neq) state, no difference form: this is the plain
 * formula against which the re-cast update of fv_substep_q is checked. */
void orc_fv_substep_literal(int n, const int *rowptr, const int *col, const double *sx, const double *sy,
                            const double *cc, double dt, double tau_u, const double *g, double *gnew)
{
    double *eq = malloc(((size_t)n * 9 + 1) * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int p = 0; p < n; p++) {
        double rho, ux, uy;
        orc_moments(g + 9 * (size_t)p, &rho, &ux, &uy);
        orc_feq(rho, ux, uy, eq + 9 * (size_t)p);
    }
#pragma omp parallel for schedule(static)
    for (int p = 0; p < n; p++)
        for (int i = 0; i < 9; i++) {
            double stream = 0.0, coll = 0.0;
            for (int e = rowptr[p]; e < rowptr[p + 1]; e++) {
                const int k = col[e];
                const double S = CX[i] * sx[e] + CY[i] * sy[e];
                stream += S * g[9 * (size_t)k + i];
                coll += cc[e] * (g[9 * (size_t)k + i] - eq[9 * (size_t)k + i]);
            }
            gnew[9 * (size_t)p + i] = g[9 * (size_t)p + i] + dt * stream - (dt / tau_u) * coll;
        }
    free(eq);
}

/* Test driver for a channel of the triangular mesh: nsteps sub-steps of the
 * solver's own update (fv_substep_q, as in the coupled step) on populations
 * g[n][9], each followed by a uniform body force (Fx, Fy) per unit volume,
 * added as the source dt F_i with F_i = 3 w_i c_i . F (zero mass, momentum
 * dt F, zero second moment), and by the wall rule (u <- 0) on the nodes with
 * wall[p] != 0.  The body force is not part of the paper's method; it drives
 * the Poiseuille check of Eq. 3 and the wall rule. */
void orc_fv_channel_run(int n, const int *rowptr, const int *col, const double *sx, const double *sy,
                        const double *cc, double dt, double tau_u, const unsigned char *wall, double Fx,
                        double Fy, int nsteps, double *g)
{
    double *q = calloc((size_t)n * 12 + 1, sizeof(double)), *qn = calloc((size_t)n * 12 + 1, sizeof(double));
    for (int p = 0; p < n; p++) state_q(g + 9 * (size_t)p, q + 12 * (size_t)p);
    for (int s = 0; s < nsteps; s++) {
        fv_substep_q(n, rowptr, col, sx, sy, cc, dt, tau_u, q, qn);
        for (int p = 0; p < n; p++) {
            double *qo = qn + 12 * (size_t)p, u1x, u1y, dfe[9];
            u1x = qo[1] + dt * Fx / qo[0];
            u1y = qo[2] + dt * Fy / qo[0];
            if (wall[p]) { u1x = 0.0; u1y = 0.0; }
            orc_feq_diff(qo[0], u1x, u1y, qo[0], qo[1], qo[2], dfe);
            for (int i = 0; i < 9; i++) {
                double Fi = wall[p] ? 0.0 : 3.0 * WQ[i] * (CX[i] * Fx + CY[i] * Fy);
                qo[3 + i] += (wall[p] ? 0.0 : dt * Fi - dfe[i]);
            }
            qo[1] = u1x;
            qo[2] = u1y;
            neq_constrain(qo);
        }
        double *t = q; q = qn; qn = t;
    }
    for (int p = 0; p < n; p++) from_q(q + 12 * (size_t)p, 1.0, g + 9 * (size_t)p);
    free(q);
    free(qn);
}

/* Test driver for the lattice: Eq. 1 on an nx x ny channel, periodic in x,
 * with stationary walls half-way between rows (below y = 0 and above
 * y = ny - 1, "half-way bounce-back": a population that would leave through
 * a wall returns reversed to the node it left) and a uniform body force Fx
 * in x (Guo, Zheng and Shi's forcing: velocity u = (sum c f + F/2) / rho in
 * f^eq, source (1 - 1/(2 tau)) w_i [3 (c_i - u) + 9 (c_i . u) c_i] . F).
 * Neither the walls nor the force are part of the paper's method; they give
 * the Poiseuille check of the lattice collide-stream.  f is [ny][nx][9]. */
void orc_lattice_channel(double *f, int nx, int ny, double tau, double Fx, int nsteps)
{
    static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    size_t nn = (size_t)nx * ny;
    double *post = malloc(nn * 9 * sizeof(double));
    for (int s = 0; s < nsteps; s++) {
        for (size_t p = 0; p < nn; p++) {
            const double *fp = f + 9 * p;
            double rho = 0.0, mx = 0.0, my = 0.0, eq[9];
            for (int i = 0; i < 9; i++) { rho += fp[i]; mx += CX[i] * fp[i]; my += CY[i] * fp[i]; }
            double ux = (mx + 0.5 * Fx) / rho, uy = my / rho;
            orc_feq(rho, ux, uy, eq);
            for (int i = 0; i < 9; i++) {
                double cu = CX[i] * ux + CY[i] * uy;
                double Fi = (1.0 - 0.5 / tau) * WQ[i] * (3.0 * (CX[i] - ux) + 9.0 * cu * CX[i]) * Fx;
                post[9 * p + i] = fp[i] - (fp[i] - eq[i]) / tau + Fi;
            }
        }
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++)
                for (int i = 0; i < 9; i++) {
                    int xs = ((x - CX[i]) % nx + nx) % nx, ys = y - CY[i];
                    size_t p = (size_t)y * nx + x;
                    f[9 * p + i] = (ys < 0 || ys >= ny) ? post[9 * p + OPP[i]] : post[9 * ((size_t)ys * nx + xs) + i];
                }
    }
    free(post);
}

/* Wall rule (the paper states only "no-slip"; reading): keep the density and
 * the non-equilibrium part of the wall node, set its velocity to zero:
 * g <- f^eq(rho, 0) + (g - f^eq(rho, u)).  In the (rho, u, g^neq) state of
 * the solver this is u <- 0. */
void orc_wall_rule(double *g)
{
    double rho, ux, uy, eq[9], eq0[9];
    orc_moments(g, &rho, &ux, &uy);
    orc_feq(rho, ux, uy, eq);
    orc_feq(rho, 0.0, 0.0, eq0);
    for (int i = 0; i < 9; i++) g[i] = eq0[i] + (g[i] - eq[i]);
}

/* ------------------------------------------------ interpolation weights --- */
/* Solve the n x n system M x = b (row-major M), Gaussian elimination with
 * partial pivoting.  Returns 0, or -1 if singular. */
static int solve_dense(int n, double *M, double *b)
{
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(M[r * n + c]) > fabs(M[piv * n + c])) piv = r;
        if (M[piv * n + c] == 0.0) return -1;
        if (piv != c) {
            for (int k = 0; k < n; k++) { double t = M[c * n + k]; M[c * n + k] = M[piv * n + k]; M[piv * n + k] = t; }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; r++) {
            double m = M[r * n + c] / M[c * n + c];
            for (int k = c; k < n; k++) M[r * n + k] -= m * M[c * n + k];
            b[r] -= m * b[c];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = b[r];
        for (int k = r + 1; k < n; k++) s -= M[r * n + k] * b[k];
        b[r] = s / M[r * n + r];
    }
    return 0;
}

/* Eq. 8: second-order shape functions on six donor nodes evaluated at (x, y).
 * The weights psi_k reproduce every quadratic exactly:
 * sum_k psi_k m(x_k - x) = m(0) for m in {1, X, Y, X^2, XY, Y^2}
 * (coordinates relative to (x, y), scaled by the largest donor distance). */
int orc_quad6_weights(const double *pts, double x, double y, double *w)
{
    double h = 0.0;
    for (int k = 0; k < 6; k++) {
        double d = hypot(pts[2 * k] - x, pts[2 * k + 1] - y);
        if (d > h) h = d;
    }
    if (!(h > 0.0)) return -1;
    double M[36];
    for (int k = 0; k < 6; k++) {
        double X = (pts[2 * k] - x) / h, Y = (pts[2 * k + 1] - y) / h;
        double m[6] = {1.0, X, Y, X * X, X * Y, Y * Y};
        for (int j = 0; j < 6; j++) M[j * 6 + k] = m[j]; /* row j: monomial j over donors */
    }
    for (int j = 0; j < 6; j++) w[j] = (j == 0) ? 1.0 : 0.0;
    return solve_dense(6, M, w);
}

/* Eq. 9: biquadratic Lagrange weights on the 3x3 lattice block centred on the
 * node nearest to the point; (fx, fy) is the offset from that centre,
 * in [-1/2, 1/2].  Donor k = (b+1)*3 + (a+1) sits at offset (a, b). */
void orc_biquad9_weights(double fx, double fy, double *w)
{
    double lx[3] = {0.5 * fx * (fx - 1.0), (1.0 - fx) * (1.0 + fx), 0.5 * fx * (fx + 1.0)};
    double ly[3] = {0.5 * fy * (fy - 1.0), (1.0 - fy) * (1.0 + fy), 0.5 * fy * (fy + 1.0)};
    for (int b = 0; b < 3; b++)
        for (int a = 0; a < 3; a++) w[b * 3 + a] = lx[a] * ly[b];
}

/* ------------------------------------------------------------- forces ----- */
/* Eq. 10-11 force on the body from nodal pressure and stress (the paper
 * computes them directly at the body nodes).  Reading: traction
 * sigma . n = -(p - p0) n - Pi^neq . n with p = rho/3, p0 = 1/3 and
 * Pi^neq_ab = sum_i c_ia c_ib (g_i - g_i^eq) (the unstructured scheme has
 * nu = c_s^2 tau_u, with no half-step shift); n points from the body into the
 * fluid; the edge value is the mean of its two end nodes; edges are straight.
 * Wall edge e runs a -> b with the fluid on its left. */
static void wall_force_q(int n_edges, const int *ea, const int *eb, const double *xy, const double *qs,
                         double *F)
{
    double fx = 0.0, fy = 0.0;
    for (int e = 0; e < n_edges; e++) {
        int nodes[2] = {ea[e], eb[e]};
        double p[2], pxx[2], pxy[2], pyy[2];
        for (int s = 0; s < 2; s++) {
            const double *q = qs + 12 * (size_t)nodes[s];
            p[s] = q[0] / 3.0;
            pxx[s] = pxy[s] = pyy[s] = 0.0;
            for (int i = 0; i < 9; i++) {
                pxx[s] += CX[i] * CX[i] * q[3 + i];
                pxy[s] += CX[i] * CY[i] * q[3 + i];
                pyy[s] += CY[i] * CY[i] * q[3 + i];
            }
        }
        double dx = xy[2 * eb[e]] - xy[2 * ea[e]], dy = xy[2 * eb[e] + 1] - xy[2 * ea[e] + 1];
        double nx = -dy, ny = dx; /* left normal times length: into the fluid */
        double pm = 0.5 * (p[0] + p[1]) - 1.0 / 3.0;
        double mxx = 0.5 * (pxx[0] + pxx[1]), mxy = 0.5 * (pxy[0] + pxy[1]), myy = 0.5 * (pyy[0] + pyy[1]);
        fx += -pm * nx - (mxx * nx + mxy * ny);
        fy += -pm * ny - (mxy * nx + myy * ny);
    }
    F[0] = fx;
    F[1] = fy;
}

/* The same from populations g[n][9]. */
void orc_wall_force(int n_edges, const int *ea, const int *eb, const double *xy, const double *g, double *F)
{
    int n = 0;
    for (int e = 0; e < n_edges; e++) {
        if (ea[e] + 1 > n) n = ea[e] + 1;
        if (eb[e] + 1 > n) n = eb[e] + 1;
    }
    double *q = malloc(((size_t)n + 1) * 12 * sizeof(double));
    for (int p = 0; p < n; p++) state_q(g + 9 * (size_t)p, q + 12 * (size_t)p);
    wall_force_q(n_edges, ea, eb, xy, q, F);
    free(q);
}

/* ============================================================ the solver == */
enum { T_FLUID = 0, T_BC = 1, T_PROLONG = 2, T_COVERED = 3, T_HOLE = 4, T_INTERP = 5 };

typedef struct {
    int nx, ny, ox, oy;
    double tau;
    double *f, *post;       /* [ny*nx][9] pre-collision state and scratch */
    unsigned char *type;
    /* snapshots of (rho, u, f^neq) of this level on the band around its child box,
     * before (A) and after (B) this level's step; dense over the child's box + 1 */
    int bx0, by0, bw, bh;
    double *snapA, *snapB;
} olevel;

typedef struct {
    int L;
    olevel lv[8];
    double u0, nu, tau_u, dt_u, chord;
    double pivot[2], ca, sa;    /* mesh pose: rotation by -alpha about the pivot */
    int n_sub;
    /* mesh */
    int n, ntri, nnz;
    double *xy;
    int *tri;
    unsigned char *kind;
    int *rowptr, *col;
    double *sx, *sy, *cc, *area;
    double *g, *gnew;
    int n_ring, *ring;          /* unstructured interpolation nodes */
    int *ring_don;              /* [n_ring][9] finest-level node indices */
    double *ring_w;             /* [n_ring][9] */
    double *Q0, *Q1;            /* [n_ring][12] interpolated (rho,u,neq) at t and t+1 */
    int n_wall, *wall;
    int n_wedge, *wea, *web;
    int n_is, *is_node;         /* structured interpolation nodes (finest index) */
    int *is_don;                /* [n_is][6] mesh nodes */
    double *is_w;               /* [n_is][6] */
    int periodic0;              /* test-only: level 0 periodic, no outer rules */
    int literal_fv;             /* test-only: Eq. 3 sub-steps by orc_fv_substep_literal */
    double fv_filter;           /* strength of the odd-even filter per finest step (0: off) */
    /* force series */
    int nf, fcap;
    double *cd, *cl;
    long step;
} orc;

static void lv_q(const olevel *l, int x, int y, double *q) { state_q(l->f + 9 * ((size_t)y * l->nx + x), q); }

/* Level-0 outer conditions (Section 4: uniform velocity and zero pressure
 * gradient at the inlet, fixed pressure and zero velocity gradient at the
 * outlet, open top and bottom).  Reading: every perimeter node takes its
 * state from the nearest interior node n (coordinates clamped to the
 * interior): inlet f = f^eq(rho_n, (u0, 0)) + f^neq_n; outlet
 * f = f^eq(1, u_n) + f^neq_n; top/bottom f = f_n.  Corners take the inlet or
 * outlet rule. */
static void apply_outer_bc(orc *o)
{
    olevel *l = &o->lv[0];
    int nx = l->nx, ny = l->ny;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            if (x != 0 && x != nx - 1 && y != 0 && y != ny - 1) continue;
            int xn = x < 1 ? 1 : (x > nx - 2 ? nx - 2 : x);
            int yn = y < 1 ? 1 : (y > ny - 2 ? ny - 2 : y);
            double q[12];
            lv_q(l, xn, yn, q);
            double *fb = l->f + 9 * ((size_t)y * nx + x);
            if (x == 0) { q[1] = o->u0; q[2] = 0.0; from_q(q, 1.0, fb); }
            else if (x == nx - 1) { q[0] = 1.0; from_q(q, 1.0, fb); }
            else memcpy(fb, l->f + 9 * ((size_t)yn * nx + xn), 9 * sizeof(double));
        }
}

/* Snapshot (rho, u, f^neq) of level c on the coarse nodes its child's
 * boundary ring is interpolated from. */
static void snapshot(orc *o, int c, double *dst)
{
    olevel *l = &o->lv[c];
#pragma omp parallel for schedule(static)
    for (int yy = 0; yy < l->bh; yy++)
        for (int xx = 0; xx < l->bw; xx++) {
            int x = l->bx0 + xx, y = l->by0 + yy;
            lv_q(l, x, y, dst + 12 * ((size_t)yy * l->bw + xx));
        }
}

/* Refinement interface, coarse -> fine (Section 4 cites Filippova and Haenel;
 * reading): the boundary ring of fine level c+1 takes f = f^eq(rho, u) +
 * tau_f/(2 tau_c) f^neq, with (rho, u, f^neq) linear in time between the
 * parent's snapshots before and after its step (fraction theta) and, for
 * ring nodes midway between coarse nodes, quadratic along the ring through
 * coarse nodes X-1, X, X+1 (weights -1/8, 3/4, 3/8 at X+1/2). */
static void prolong(orc *o, int c, double theta)
{
    olevel *pc = &o->lv[c], *pf = &o->lv[c + 1];
    double scale = pf->tau / (2.0 * pc->tau);
    static const double W3[3] = {-1.0 / 8.0, 3.0 / 4.0, 3.0 / 8.0};
    for (int j = 0; j < pf->ny; j++)
        for (int i = 0; i < pf->nx; i++) {
            if (i != 0 && i != pf->nx - 1 && j != 0 && j != pf->ny - 1) continue;
            double q[12] = {0};
            int nd = 1, dx = 0, dy = 0;
            int X = pf->ox + i / 2, Y = pf->oy + j / 2; /* floor for odd index */
            if (i % 2) { nd = 3; dx = 1; X -= 1; }
            else if (j % 2) { nd = 3; dy = 1; Y -= 1; }
            for (int k = 0; k < nd; k++) {
                int x = X + k * dx, y = Y + k * dy;
                size_t s = 12 * ((size_t)(y - pc->by0) * pc->bw + (x - pc->bx0));
                double wk = nd == 1 ? 1.0 : W3[k];
                for (int m = 0; m < 12; m++)
                    q[m] += wk * ((1.0 - theta) * pc->snapA[s + m] + theta * pc->snapB[s + m]);
            }
            from_q(q, scale, pf->f + 9 * ((size_t)j * pf->nx + i));
        }
}

/* Refinement interface, fine -> coarse: every coarse node at least one coarse
 * cell inside the child box takes the coincident fine node's state with
 * f^neq rescaled by 2 tau_c / tau_f. */
static void restrict_level(orc *o, int c)
{
    olevel *pc = &o->lv[c], *pf = &o->lv[c + 1];
    double scale = 2.0 * pc->tau / pf->tau;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < pc->ny; y++)
        for (int x = 0; x < pc->nx; x++) {
            if (pc->type[(size_t)y * pc->nx + x] != T_COVERED) continue;
            double q[12];
            lv_q(pf, 2 * (x - pf->ox), 2 * (y - pf->oy), q);
            from_q(q, scale, pc->f + 9 * ((size_t)y * pc->nx + x));
        }
}

/* Eq. 9 applied to the lattice state: (rho, u, f^neq) at every unstructured
 * interpolation node, from its 9 structured donors. */
static void ring_interp(orc *o, double *Q)
{
    olevel *l = &o->lv[o->L - 1];
#pragma omp parallel for schedule(static)
    for (int r = 0; r < o->n_ring; r++) {
        double *q = Q + 12 * (size_t)r;
        for (int m = 0; m < 12; m++) q[m] = 0.0;
        for (int k = 0; k < 9; k++) {
            double qk[12];
            state_q(l->f + 9 * (size_t)o->ring_don[9 * r + k], qk);
            for (int m = 0; m < 12; m++) q[m] += o->ring_w[9 * r + k] * qk[m];
        }
    }
}

/* Eq. 5-7 interface values on the unstructured interpolation nodes at
 * fraction theta of the structured step: f^eq,s + (1 - 1/(2 tau_s)) f^neq,s. */
static void ring_set(orc *o, double theta)
{
    double tau_s = o->lv[o->L - 1].tau;
    for (int r = 0; r < o->n_ring; r++) {
        double q[12];
        for (int m = 0; m < 12; m++)
            q[m] = (1.0 - theta) * o->Q0[12 * (size_t)r + m] + theta * o->Q1[12 * (size_t)r + m];
        eq5_q(q, tau_s, o->g + 12 * (size_t)o->ring[r]);
    }
}

/* Eq. 4 with Eq. 8: post-collision state of the structured interpolation
 * nodes, from the unstructured state (rho, u, g^neq) at time t. */
static void hole_interp(orc *o)
{
    olevel *l = &o->lv[o->L - 1];
#pragma omp parallel for schedule(static)
    for (int s = 0; s < o->n_is; s++) {
        double q[12] = {0};
        for (int k = 0; k < 6; k++) {
            const double *qk = o->g + 12 * (size_t)o->is_don[6 * s + k];
            for (int m = 0; m < 12; m++) q[m] += o->is_w[6 * s + k] * qk[m];
        }
        orc_eq4_post(q, l->tau, l->post + 9 * (size_t)o->is_node[s]);
    }
}

/* Eq. 1 on level c: collide every computed node, give the structured
 * interpolation nodes their Eq. 4 state, stream by pulling from x - c_i. */
static void collide_stream(orc *o, int c)
{
    olevel *l = &o->lv[c];
    size_t nn = (size_t)l->nx * l->ny;
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < nn; p++) {
        double *dst = l->post + 9 * p;
        if (l->type[p] == T_HOLE || l->type[p] == T_INTERP) {
            for (int i = 0; i < 9; i++) dst[i] = NAN;
            continue;
        }
        memcpy(dst, l->f + 9 * p, 9 * sizeof(double));
        orc_bgk_collide(dst, l->tau);
    }
    if (c == o->L - 1 && o->n) hole_interp(o);
    stream_pull(l->post, l->f, l->nx, l->ny, c == 0 && o->periodic0);
}

/* Test-only alternative to fv_substep_q inside the solver: the state g (as
 * (rho, u, g^neq)) is turned into populations, advanced by the literal Eq. 3
 * and turned back, into gnew. */
static void fv_substep_pop(orc *o)
{
    const size_t n = (size_t)o->n;
    double *a = malloc((9 * n + 1) * sizeof(double)), *b = malloc((9 * n + 1) * sizeof(double));
    for (size_t p = 0; p < n; p++) from_q(o->g + 12 * p, 1.0, a + 9 * p);
    orc_fv_substep_literal(o->n, o->rowptr, o->col, o->sx, o->sy, o->cc, o->dt_u, o->tau_u, a, b);
    for (size_t p = 0; p < n; p++) state_q(b + 9 * p, o->gnew + 12 * p);
    free(a);
    free(b);
}

/* Odd-even filter of the mesh state, once per finest step after the Eq. 3
 * sub-steps, when o->fv_filter = sigma > 0 (an addition to the paper's method,
 * off by default).  With the graph Laplacian of the Eq. 3 collision weights,
 *   (L g)_i(P) = sum_{k != P} C_Pk [g_i(P_k) - g_i(P)],
 * every population of every fluid node takes one step of a biharmonic
 * (fourth-order) damping,
 *   g_i(P) <- g_i(P) - sigma (L d)_i(P),  d = L g at fluid nodes, 0 elsewhere;
 * wall and outer-ring nodes are left as they are (at a boundary node L is a
 * one-sided, first-order difference, which would act on the wall pressure and
 * stress).  A_P C_Pk is symmetric in (P, k) (both are 7/108 of the two
 * triangles' areas at edge Pk), so on a mesh without boundary nodes L and the
 * filter conserve mass and momentum exactly.  On smooth fields the filter is a
 * hyper-diffusion
 * of O(sigma h^4 k^4) per step; on the node-to-node (odd-even) oscillations,
 * which the central fluxes of Eq. 3 neither advect nor damp, L has an
 * eigenvalue of order one and the filter damps them at O(sigma) per step.
 * The first Laplacian is formed on the (rho, u, g^neq) state as
 * fv_substep_q forms its differences; the second on the stored differences. */
static void fv_lap_q(int n, const int *rowptr, const int *col, const double *cc, const unsigned char *kind,
                     const double *q, double *d)
{
#pragma omp parallel for schedule(static)
    for (int p = 0; p < n; p++) {
        const double *qp = q + 12 * (size_t)p;
        double acc[9] = {0};
        if (kind && kind[p] != 0) {
            for (int i = 0; i < 9; i++) d[9 * (size_t)p + i] = 0.0;
            continue;
        }
        for (int e = rowptr[p]; e < rowptr[p + 1]; e++) {
            const int k = col[e];
            if (k == p) continue;
            const double *qk = q + 12 * (size_t)k;
            double dfe[9];
            orc_feq_diff(qk[0], qk[1], qk[2], qp[0], qp[1], qp[2], dfe);
            for (int i = 0; i < 9; i++) acc[i] += cc[e] * (dfe[i] + qk[3 + i] - qp[3 + i]);
        }
        for (int i = 0; i < 9; i++) d[9 * (size_t)p + i] = acc[i];
    }
}

static void fv_filter_q(int n, const int *rowptr, const int *col, const double *cc, const unsigned char *kind,
                        double sigma, const double *q, double *qn)
{
    double *d = malloc(((size_t)n * 9 + 1) * sizeof(double));
    fv_lap_q(n, rowptr, col, cc, kind, q, d);
#pragma omp parallel for schedule(static)
    for (int p = 0; p < n; p++) {
        const double *qp = q + 12 * (size_t)p, *dp = d + 9 * (size_t)p;
        double acc[9] = {0};
        if (kind && kind[p] != 0) {
            memcpy(qn + 12 * (size_t)p, qp, 12 * sizeof(double));
            continue;
        }
        for (int e = rowptr[p]; e < rowptr[p + 1]; e++) {
            const int k = col[e];
            if (k == p) continue;
            for (int i = 0; i < 9; i++) acc[i] += cc[e] * (d[9 * (size_t)k + i] - dp[i]);
        }
        double drho = 0.0, djx = 0.0, djy = 0.0;
        for (int i = 0; i < 9; i++) {
            acc[i] *= -sigma;
            drho += acc[i];
            djx += CX[i] * acc[i];
            djy += CY[i] * acc[i];
        }
        double *qo = qn + 12 * (size_t)p;
        const double rho = qp[0] + drho;
        qo[0] = rho;
        qo[1] = qp[1] + (djx - drho * qp[1]) / rho;
        qo[2] = qp[2] + (djy - drho * qp[2]) / rho;
        double dfe[9];
        orc_feq_diff(qo[0], qo[1], qo[2], qp[0], qp[1], qp[2], dfe);
        for (int i = 0; i < 9; i++) qo[3 + i] = qp[3 + i] + acc[i] - dfe[i];
        neq_constrain(qo);
    }
    free(d);
}

static void fv_filter(orc *o)
{
    fv_filter_q(o->n, o->rowptr, o->col, o->cc, o->kind, o->fv_filter, o->g, o->gnew);
    double *t = o->g; o->g = o->gnew; o->gnew = t;
}

/* The filter on populations g[n][9] -> gnew (kind may be NULL: no wall nodes). */
void orc_fv_filter(int n, const int *rowptr, const int *col, const double *cc, const unsigned char *kind,
                   double sigma, const double *g, double *gnew)
{
    double *q = calloc((size_t)n * 12 + 1, sizeof(double)), *qn = calloc((size_t)n * 12 + 1, sizeof(double));
    for (int p = 0; p < n; p++) state_q(g + 9 * (size_t)p, q + 12 * (size_t)p);
    fv_filter_q(n, rowptr, col, cc, kind, sigma, q, qn);
    for (int p = 0; p < n; p++) from_q(qn + 12 * (size_t)p, 1.0, gnew + 9 * (size_t)p);
    free(q);
    free(qn);
}

/* One step of the finite-volume part (H4 of the coupling): n sub-steps of
 * Eq. 3 on all mesh nodes, the interface nodes first set by Eq. 5-7 and the
 * wall rule applied after each sub-step. */
static void fv_steps(orc *o)
{
    for (int m = 0; m < o->n_sub; m++) {
        ring_set(o, (double)m / o->n_sub);
        if (o->literal_fv) fv_substep_pop(o);
        else fv_substep_q(o->n, o->rowptr, o->col, o->sx, o->sy, o->cc, o->dt_u, o->tau_u, o->g, o->gnew);
        for (int w = 0; w < o->n_wall; w++) {  /* wall rule: u <- 0, rho and g^neq kept */
            o->gnew[12 * (size_t)o->wall[w] + 1] = 0.0;
            o->gnew[12 * (size_t)o->wall[w] + 2] = 0.0;
        }
        double *t = o->g; o->g = o->gnew; o->gnew = t;
    }
    if (o->fv_filter > 0.0) fv_filter(o);
}

/* One step of level c (its own clock).  theta_next: parent-time fraction
 * reached at the end of this step, used to refill the boundary ring. */
static void level_step(orc *o, int c, double theta_next)
{
    int finest = (c == o->L - 1);
    if (finest && o->n) ring_interp(o, o->Q0);
    collide_stream(o, c);
    if (c == 0) { if (!o->periodic0) apply_outer_bc(o); }
    else prolong(o, c - 1, theta_next);
    if (finest && o->n) {
        ring_interp(o, o->Q1);
        fv_steps(o);
    }
}

static void advance(orc *o, int c, double theta_next)
{
    if (c < o->L - 1) snapshot(o, c, o->lv[c].snapA);
    level_step(o, c, theta_next);
    if (c < o->L - 1) {
        snapshot(o, c, o->lv[c].snapB);
        advance(o, c + 1, 0.5);
        advance(o, c + 1, 1.0);
        restrict_level(o, c);
    }
}

/* Mean pressure and skin-friction coefficients (Eq. 12-13), per wall node.
 * Node P carries N_P = half the sum of its wall edges' normals times length
 * (into the fluid), so that the wall force above is exactly
 *   sum_P [-(p_P - p0) N_P - Pi^neq_P N_P]
 * with p = rho / 3 and p0 = 1/3.  With n = N_P / |N_P| and s the unit tangent
 * pointing downstream along the chord, the viscous traction -Pi^neq n splits
 * into a normal part c_n n and the wall shear stress tau_w s.  Per wall node
 * (ascending node index) out[10] = (x/C along the chord from the leading
 * edge, side (+1 upper, -1 lower surface), C_p, C_f = tau_w / q, C_n = c_n / q,
 * |N_P|, n_x, n_y, s_x, s_y) with q = rho0 u0^2 / 2, rho0 = 1.  Returns the
 * number of wall nodes (out may be NULL to query it). */
int orc_wall_coeffs(const orc *o, double *out)
{
    int nw = 0;
    for (int p = 0; p < o->n; p++) nw += o->kind[p] == 1;
    if (!out || nw == 0) return nw;
    double *N = calloc((size_t)o->n * 2, sizeof(double));
    for (int e = 0; e < o->n_wedge; e++) {
        int a = o->wea[e], b = o->web[e];
        double dx = o->xy[2 * b] - o->xy[2 * a], dy = o->xy[2 * b + 1] - o->xy[2 * a + 1];
        N[2 * a] += -0.5 * dy; N[2 * a + 1] += 0.5 * dx;
        N[2 * b] += -0.5 * dy; N[2 * b + 1] += 0.5 * dx;
    }
    double q = 0.5 * o->u0 * o->u0;
    double chx = o->ca, chy = -o->sa; /* body chord direction in the lattice frame */
    int k = 0;
    for (int p = 0; p < o->n; p++) {
        if (o->kind[p] != 1) continue;
        const double *g = o->g + 12 * (size_t)p;  /* rho, u, f^neq */
        double pxx = 0.0, pxy = 0.0, pyy = 0.0;
        for (int i = 0; i < 9; i++) {
            pxx += CX[i] * CX[i] * g[3 + i];
            pxy += CX[i] * CY[i] * g[3 + i];
            pyy += CY[i] * CY[i] * g[3 + i];
        }
        double A = sqrt(N[2 * p] * N[2 * p] + N[2 * p + 1] * N[2 * p + 1]);
        double nx = N[2 * p] / A, ny = N[2 * p + 1] / A;
        double sx = -ny, sy = nx;
        if (sx * chx + sy * chy < 0.0) { sx = -sx; sy = -sy; }
        double tx = -(pxx * nx + pxy * ny), ty = -(pxy * nx + pyy * ny);
        /* body-frame position: undo the rotation about the pivot (quarter chord) */
        double dx = o->xy[2 * p] - o->pivot[0], dy = o->xy[2 * p + 1] - o->pivot[1];
        double xb = o->ca * dx - o->sa * dy, yb = o->sa * dx + o->ca * dy;
        double *r = out + 10 * (size_t)k++;
        r[0] = xb / o->chord + 0.25;
        r[1] = yb >= 0.0 ? 1.0 : -1.0;
        r[2] = (g[0] - 1.0) / 3.0 / q;
        r[3] = (tx * sx + ty * sy) / q;
        r[4] = (tx * nx + ty * ny) / q;
        r[5] = A;
        r[6] = nx; r[7] = ny; r[8] = sx; r[9] = sy;
    }
    free(N);
    return nw;
}

static void record_forces(orc *o)
{
    if (!o->n) return;
    double F[2];
    wall_force_q(o->n_wedge, o->wea, o->web, o->xy, o->g, F);
    double qdyn = 0.5 * o->u0 * o->u0 * o->chord;
    if (o->nf == o->fcap) {
        o->fcap = o->fcap ? 2 * o->fcap : 1024;
        o->cd = realloc(o->cd, (size_t)o->fcap * sizeof(double));
        o->cl = realloc(o->cl, (size_t)o->fcap * sizeof(double));
    }
    o->cd[o->nf] = F[0] / qdyn;
    o->cl[o->nf] = F[1] / qdyn;
    o->nf++;
}

/* Test functional for the adjoint of the finite-volume part: from the current
 * mesh state, n_window sub-steps as in fv_steps (Eq. 3 on every node, then
 * the wall rule), except that the interface rows take the Eq. 5-7 state of
 * one fixed set of Eq. 9 data, that of the current lattice, and that they are
 * set after every sub-step but the last of a finest step (so the window
 * starts from the interface rows as they are); then Eq. 10-11 of the final
 * state, J = (wd F_x + wl F_y) / (1/2 u0^2 C).  Perturbations for finite
 * differences: the initial populations by hg dg ([n][9], input node order),
 * the operator entries (s_x, s_y, C) by hc dcoef ([nnz][3], CSR order), and
 * the geometry: the input-frame node coordinates by hx dxy ([n][2]) and the
 * angle of attack by daoa degrees, after which the pose, the Eq. 3
 * operators and the wall normals are rebuilt (the state and the interface
 * data stay as they are), each when given.  The oracle's own state is not
 * changed.  Returns 0, or -1 without a mesh, with n_window outside
 * 1..n_sub, or if the moved mesh has an inverted triangle. */
int orc_fv_window(orc *o, int n_window, double wd, double wl, const double *dg, double hg, const double *dcoef,
                  double hc, const double *dxy, double hx, double daoa, double *J)
{
    if (!o->n || n_window < 1 || n_window > o->n_sub) return -1;
    const size_t n = (size_t)o->n, nnz = (size_t)o->nnz;
    double *q = malloc(12 * n * sizeof(double)), *qn = malloc(12 * n * sizeof(double));
    double *sx = malloc(nnz * sizeof(double)), *sy = malloc(nnz * sizeof(double)), *cc = malloc(nnz * sizeof(double));
    double *Q = malloc(((size_t)o->n_ring * 12 + 1) * sizeof(double));
    double *xy = malloc(2 * n * sizeof(double));
    memcpy(xy, o->xy, 2 * n * sizeof(double));
    memcpy(sx, o->sx, nnz * sizeof(double));
    memcpy(sy, o->sy, nnz * sizeof(double));
    memcpy(cc, o->cc, nnz * sizeof(double));
    if (dxy || daoa != 0.0) {
        /* back to the input frame (rotation by +alpha about the pivot), move,
         * and pose again at alpha + daoa */
        const double al = atan2(o->sa, o->ca) + daoa * M_PI / 180.0, c2 = cos(al), s2 = sin(al);
        for (size_t p = 0; p < n; p++) {
            const double dx = o->xy[2 * p] - o->pivot[0], dy = o->xy[2 * p + 1] - o->pivot[1];
            double xb = o->ca * dx - o->sa * dy, yb = o->sa * dx + o->ca * dy;
            if (dxy) { xb += hx * dxy[2 * p]; yb += hx * dxy[2 * p + 1]; }
            xy[2 * p] = o->pivot[0] + (c2 * xb + s2 * yb);
            xy[2 * p + 1] = o->pivot[1] + (c2 * yb - s2 * xb);
        }
        int *rp2 = malloc((n + 1) * sizeof(int)), *col2 = malloc((n + 6 * (size_t)o->ntri) * sizeof(int));
        double *b1 = malloc((n + 6 * (size_t)o->ntri) * sizeof(double)), *b2 = malloc((n + 6 * (size_t)o->ntri) * sizeof(double));
        double *b3 = malloc((n + 6 * (size_t)o->ntri) * sizeof(double)), *ar = malloc(n * sizeof(double));
        int nz = orc_fv_operators(o->n, xy, o->ntri, o->tri, NULL, rp2, col2, b1, b2, b3, ar);
        int same = nz == o->nnz;
        for (size_t e = 0; same && e < nnz; e++) same = col2[e] == o->col[e];
        if (same) {
            memcpy(sx, b1, nnz * sizeof(double));
            memcpy(sy, b2, nnz * sizeof(double));
            memcpy(cc, b3, nnz * sizeof(double));
        }
        free(rp2); free(col2); free(b1); free(b2); free(b3); free(ar);
        if (!same) {
            free(q); free(qn); free(sx); free(sy); free(cc); free(Q); free(xy);
            return -1;
        }
    }
    memcpy(q, o->g, 12 * n * sizeof(double));
    if (dg) {
        for (size_t p = 0; p < n; p++) {
            double f[9];
            from_q(q + 12 * p, 1.0, f);
            for (int i = 0; i < 9; i++) f[i] += hg * dg[9 * p + i];
            state_q(f, q + 12 * p);
        }
    }
    for (size_t e = 0; dcoef && e < nnz; e++) {
        sx[e] += hc * dcoef[3 * e];
        sy[e] += hc * dcoef[3 * e + 1];
        cc[e] += hc * dcoef[3 * e + 2];
    }
    ring_interp(o, Q);
    const double tau_s = o->lv[o->L - 1].tau;
    for (int m = 0; m < n_window; m++) {
        fv_substep_q(o->n, o->rowptr, o->col, sx, sy, cc, o->dt_u, o->tau_u, q, qn);
        for (int w = 0; w < o->n_wall; w++) {
            qn[12 * (size_t)o->wall[w] + 1] = 0.0;
            qn[12 * (size_t)o->wall[w] + 2] = 0.0;
        }
        if (m < o->n_sub - 1)
            for (int r = 0; r < o->n_ring; r++) eq5_q(Q + 12 * (size_t)r, tau_s, qn + 12 * (size_t)o->ring[r]);
        double *t = q; q = qn; qn = t;
    }
    double F[2];
    wall_force_q(o->n_wedge, o->wea, o->web, xy, q, F);
    *J = (wd * F[0] + wl * F[1]) / (0.5 * o->u0 * o->u0 * o->chord);
    free(q); free(qn); free(sx); free(sy); free(cc); free(Q); free(xy);
    return 0;
}

void orc_step(orc *o, int ncoarse)
{
    for (int s = 0; s < ncoarse; s++) {
        advance(o, 0, 0.0);
        record_forces(o);
        o->step++;
    }
}

/* ------------------------------------------------------------ set-up ----- */
static void set_err(char *err, int len, const char *msg)
{
    if (err && len > 0) { strncpy(err, msg, (size_t)len - 1); err[len - 1] = 0; }
}

void orc_destroy(orc *o)
{
    if (!o) return;
    for (int c = 0; c < o->L; c++) {
        free(o->lv[c].f); free(o->lv[c].post); free(o->lv[c].type);
        free(o->lv[c].snapA); free(o->lv[c].snapB);
    }
    free(o->xy); free(o->tri); free(o->kind); free(o->rowptr); free(o->col);
    free(o->sx); free(o->sy); free(o->cc); free(o->area); free(o->g); free(o->gnew);
    free(o->ring); free(o->ring_don); free(o->ring_w); free(o->Q0); free(o->Q1);
    free(o->wall); free(o->wea); free(o->web); free(o->is_node); free(o->is_don); free(o->is_w);
    free(o->cd); free(o->cl);
    free(o);
}

/* Finite-volume sub-steps per structured step when the caller passes 0.
 * The paper uses n = 10; reading: at least 10, and enough that the explicit
 * (forward Euler) update of Eq. 3 is stable.  A mode damped at rate
 * a = 1/tau_u and oscillating at b = sqrt(2) max_P sum_k |s_Pk| (|c| <= sqrt(2))
 * is stable for dt_u <= 2a / (a^2 + b^2); a safety factor 1.1 is applied:
 * n = max(10, ceil(1.1 (a^2 + b^2) / (2a))). */
static int auto_n_sub(const orc *o)
{
    double smax = 0.0;
    for (int p = 0; p < o->n; p++) {
        double sum = 0.0;
        for (int e = o->rowptr[p]; e < o->rowptr[p + 1]; e++) sum += hypot(o->sx[e], o->sy[e]);
        if (sum > smax) smax = sum;
    }
    double a = 1.0 / o->tau_u, b = sqrt(2.0) * smax;
    double n = ceil(1.1 * (a * a + b * b) / (2.0 * a));
    return n < 10.0 ? 10 : (int)n;
}

orc *orc_create(int L, const int *levels, int n, const double *xy, int ntri, const int *tri,
                const unsigned char *kind, double chord, const double *pivot, const double *hole,
                double Re, double Ma, double aoa_deg, int n_sub, uint64_t seed, double perturb,
                int flags, char *err, int errlen)
{
    if (L < 1 || L > 8) { set_err(err, errlen, "level count out of range"); return NULL; }
    orc *o = calloc(1, sizeof(orc));
    o->L = L;
    o->periodic0 = flags & 1;
    o->literal_fv = (flags & 2) != 0;
    o->chord = chord;
    o->u0 = Ma / sqrt(3.0);
    o->nu = o->u0 * chord / Re;
    /* finest level: nu = (tau_s - 1/2)/3; level c: tau_c - 1/2 = (tau_s - 1/2) / 2^(L-1-c) */
    for (int c = 0; c < L; c++) {
        olevel *l = &o->lv[c];
        l->nx = levels[4 * c]; l->ny = levels[4 * c + 1]; l->ox = levels[4 * c + 2]; l->oy = levels[4 * c + 3];
        l->tau = 0.5 + 3.0 * o->nu / (double)(1 << (L - 1 - c));
        if (l->nx < 4 || l->ny < 4) { set_err(err, errlen, "level too small"); orc_destroy(o); return NULL; }
        if (c > 0 && (l->nx % 2 == 0 || l->ny % 2 == 0)) { set_err(err, errlen, "refined level needs odd node counts"); orc_destroy(o); return NULL; }
        size_t nn = (size_t)l->nx * l->ny;
        l->f = malloc(nn * 9 * sizeof(double));
        l->post = malloc(nn * 9 * sizeof(double));
        l->type = calloc(nn, 1);
    }
    o->tau_u = 3.0 * o->nu; /* nu = c_s^2 tau_u */
    for (int c = 1; c < L; c++) {
        olevel *pc = &o->lv[c - 1], *pf = &o->lv[c];
        int mx = (pf->nx - 1) / 2, my = (pf->ny - 1) / 2;
        if (pf->ox < 2 || pf->oy < 2 || pf->ox + mx > pc->nx - 3 || pf->oy + my > pc->ny - 3) {
            set_err(err, errlen, "refined box must sit at least two nodes inside its parent");
            orc_destroy(o); return NULL;
        }
        pc->bx0 = pf->ox - 1; pc->by0 = pf->oy - 1; pc->bw = mx + 2; pc->bh = my + 2;
        pc->snapA = malloc((size_t)pc->bw * pc->bh * 12 * sizeof(double));
        pc->snapB = malloc((size_t)pc->bw * pc->bh * 12 * sizeof(double));
        for (int y = pf->oy + 1; y <= pf->oy + my - 1; y++)
            for (int x = pf->ox + 1; x <= pf->ox + mx - 1; x++) pc->type[(size_t)y * pc->nx + x] = T_COVERED;
    }
    for (int c = 0; c < L; c++) {
        olevel *l = &o->lv[c];
        for (int y = 0; y < l->ny; y++)
            for (int x = 0; x < l->nx; x++)
                if (x == 0 || y == 0 || x == l->nx - 1 || y == l->ny - 1)
                    l->type[(size_t)y * l->nx + x] = c == 0 ? T_BC : T_PROLONG;
    }

    /* mesh: rotate by -alpha about the pivot (positive alpha = nose up) */
    double al = aoa_deg * M_PI / 180.0, ca = cos(al), sa = sin(al);
    o->pivot[0] = pivot[0];
    o->pivot[1] = pivot[1];
    o->ca = ca;
    o->sa = sa;
    o->n = n;
    o->ntri = ntri;
    olevel *lf = &o->lv[L - 1];
    if (n > 0) {
        o->xy = malloc((size_t)n * 2 * sizeof(double));
        for (int p = 0; p < n; p++) {
            double dx = xy[2 * p] - pivot[0], dy = xy[2 * p + 1] - pivot[1];
            o->xy[2 * p] = pivot[0] + (ca * dx + sa * dy);
            o->xy[2 * p + 1] = pivot[1] + (ca * dy - sa * dx);
        }
        o->tri = malloc((size_t)ntri * 3 * sizeof(int));
        memcpy(o->tri, tri, (size_t)ntri * 3 * sizeof(int));
        o->kind = malloc((size_t)n);
        memcpy(o->kind, kind, (size_t)n);
        int cap = n + 6 * ntri;
        o->rowptr = malloc(((size_t)n + 1) * sizeof(int));
        o->col = malloc((size_t)cap * sizeof(int));
        o->sx = malloc((size_t)cap * sizeof(double));
        o->sy = malloc((size_t)cap * sizeof(double));
        o->cc = malloc((size_t)cap * sizeof(double));
        o->area = malloc((size_t)n * sizeof(double));
        o->nnz = orc_fv_operators(n, o->xy, ntri, o->tri, NULL, o->rowptr, o->col, o->sx, o->sy, o->cc, o->area);
        if (o->nnz < 0) { set_err(err, errlen, "degenerate or inverted triangle"); orc_destroy(o); return NULL; }
        o->n_sub = n_sub > 0 ? n_sub : auto_n_sub(o);
        o->dt_u = 1.0 / o->n_sub;
        o->g = malloc((size_t)n * 12 * sizeof(double));     /* (rho, u, g^neq) per node */
        o->gnew = malloc((size_t)n * 12 * sizeof(double));
        /* node lists */
        o->ring = malloc((size_t)n * sizeof(int));
        o->wall = malloc((size_t)n * sizeof(int));
        for (int p = 0; p < n; p++) {
            if (kind[p] == 2) o->ring[o->n_ring++] = p;
            if (kind[p] == 1) o->wall[o->n_wall++] = p;
        }
        /* wall edges: boundary edges with two wall end nodes, oriented as in
         * their (counter-clockwise) triangle */
        o->wea = malloc((size_t)3 * ntri * sizeof(int));
        o->web = malloc((size_t)3 * ntri * sizeof(int));
        oedge *et = edge_table(ntri, tri);
        for (int t = 0; t < ntri; t++)
            for (int a = 0; a < 3; a++) {
                int ia = tri[3 * t + a], ib = tri[3 * t + (a + 1) % 3];
                if (kind[ia] != 1 || kind[ib] != 1) continue;
                if (!edge_find(et, ntri, ib, ia)) { o->wea[o->n_wedge] = ia; o->web[o->n_wedge] = ib; o->n_wedge++; }
            }
        /* structured activity on the finest level: inside the hole ellipse
         * (rotated with the body) is not computed */
        for (int y = 0; y < lf->ny; y++)
            for (int x = 0; x < lf->nx; x++) {
                double dx = (double)x - pivot[0], dy = (double)y - pivot[1];
                double X = (ca * dx - sa * dy) + pivot[0] - hole[0];
                double Y = (sa * dx + ca * dy) + pivot[1] - hole[1];
                double qx = X / hole[2], qy = Y / hole[3];
                if (qx * qx + qy * qy < 1.0) {
                    size_t p = (size_t)y * lf->nx + x;
                    if (lf->type[p] != T_FLUID) { free(et); set_err(err, errlen, "hole reaches a level boundary"); orc_destroy(o); return NULL; }
                    lf->type[p] = T_HOLE;
                }
            }
        /* structured interpolation nodes: hole nodes with a computed D2Q9 neighbour */
        size_t nnf = (size_t)lf->nx * lf->ny;
        o->is_node = malloc(nnf * sizeof(int));
        for (int y = 1; y < lf->ny - 1; y++)
            for (int x = 1; x < lf->nx - 1; x++) {
                size_t p = (size_t)y * lf->nx + x;
                if (lf->type[p] != T_HOLE) continue;
                int near = 0;
                for (int i = 1; i < 9; i++) {
                    unsigned char t = lf->type[(size_t)(y + CY[i]) * lf->nx + x + CX[i]];
                    if (t != T_HOLE && t != T_INTERP) near = 1;
                }
                if (near) o->is_node[o->n_is++] = (int)p;
            }
        for (int s = 0; s < o->n_is; s++) lf->type[o->is_node[s]] = T_INTERP;
        /* a covered coarse node whose coincident finer node is not computed
         * (hole or interpolation node) is not computed either */
        for (int c = L - 2; c >= 0; c--) {
            olevel *pc = &o->lv[c], *pf = &o->lv[c + 1];
            for (int y = 0; y < pc->ny; y++)
                for (int x = 0; x < pc->nx; x++) {
                    size_t p = (size_t)y * pc->nx + x;
                    if (pc->type[p] != T_COVERED) continue;
                    unsigned char t = pf->type[(size_t)(2 * (y - pf->oy)) * pf->nx + 2 * (x - pf->ox)];
                    if (t == T_HOLE || t == T_INTERP) pc->type[p] = T_HOLE;
                }
        }
        /* Eq. 8 stencils: the triangle holding the node (lowest index if on an
         * edge) plus the far vertex of each of its three edge neighbours */
        o->is_don = malloc((size_t)o->n_is * 6 * sizeof(int));
        o->is_w = malloc((size_t)o->n_is * 6 * sizeof(double));
        for (int s = 0; s < o->n_is; s++) {
            int p = o->is_node[s];
            double x = (double)(p % lf->nx), y = (double)(p / lf->nx);
            int found = -1;
            for (int t = 0; t < ntri && found < 0; t++) {
                const double *a = o->xy + 2 * tri[3 * t], *b = o->xy + 2 * tri[3 * t + 1], *c = o->xy + 2 * tri[3 * t + 2];
                double s0 = (b[0] - x) * (c[1] - y) - (b[1] - y) * (c[0] - x);
                double s1 = (c[0] - x) * (a[1] - y) - (c[1] - y) * (a[0] - x);
                double s2 = (a[0] - x) * (b[1] - y) - (a[1] - y) * (b[0] - x);
                if (s0 >= 0.0 && s1 >= 0.0 && s2 >= 0.0) found = t;
            }
            if (found < 0) { free(et); set_err(err, errlen, "structured interpolation node outside the mesh"); orc_destroy(o); return NULL; }
            int *d = o->is_don + 6 * s;
            for (int a = 0; a < 3; a++) d[a] = tri[3 * found + a];
            for (int a = 0; a < 3; a++) {
                int e0 = tri[3 * found + (a + 1) % 3], e1 = tri[3 * found + (a + 2) % 3];
                const oedge *nb = edge_find(et, ntri, e1, e0);
                if (!nb) { free(et); set_err(err, errlen, "interpolation triangle touches the mesh boundary"); orc_destroy(o); return NULL; }
                d[3 + a] = nb->far;
            }
            double pts[12];
            for (int k = 0; k < 6; k++) { pts[2 * k] = o->xy[2 * d[k]]; pts[2 * k + 1] = o->xy[2 * d[k] + 1]; }
            if (orc_quad6_weights(pts, x, y, o->is_w + 6 * s)) { free(et); set_err(err, errlen, "singular 6-node stencil"); orc_destroy(o); return NULL; }
        }
        free(et);
        /* Eq. 9 stencils of the unstructured interpolation nodes */
        o->ring_don = malloc((size_t)o->n_ring * 9 * sizeof(int));
        o->ring_w = malloc((size_t)o->n_ring * 9 * sizeof(double));
        o->Q0 = malloc((size_t)o->n_ring * 12 * sizeof(double));
        o->Q1 = malloc((size_t)o->n_ring * 12 * sizeof(double));
        for (int r = 0; r < o->n_ring; r++) {
            double x = o->xy[2 * o->ring[r]], y = o->xy[2 * o->ring[r] + 1];
            int X0 = (int)floor(x + 0.5), Y0 = (int)floor(y + 0.5);
            orc_biquad9_weights(x - X0, y - Y0, o->ring_w + 9 * r);
            for (int b = -1; b <= 1; b++)
                for (int a = -1; a <= 1; a++) {
                    int X = X0 + a, Y = Y0 + b;
                    if (X < 0 || Y < 0 || X >= lf->nx || Y >= lf->ny) { set_err(err, errlen, "ring donor outside the finest level"); orc_destroy(o); return NULL; }
                    size_t p = (size_t)Y * lf->nx + X;
                    if (lf->type[p] == T_HOLE || lf->type[p] == T_INTERP) { set_err(err, errlen, "ring donor inside the hole"); orc_destroy(o); return NULL; }
                    o->ring_don[9 * r + (b + 1) * 3 + (a + 1)] = (int)p;
                }
        }
    } else {
        o->n_sub = 0;
    }

    /* initial state: rho = 1 + perturb * xi, u = (u0, 0) (zero at wall nodes) */
    for (int c = 0; c < L; c++) {
        olevel *l = &o->lv[c];
        size_t nn = (size_t)l->nx * l->ny;
        for (size_t p = 0; p < nn; p++) {
            double rho = 1.0 + perturb * orc_uniform(seed, (uint64_t)c, p);
            orc_feq(rho, o->u0, 0.0, l->f + 9 * p);
            if (l->type[p] == T_HOLE || l->type[p] == T_INTERP)
                for (int i = 0; i < 9; i++) l->f[9 * p + i] = NAN;
        }
    }
    for (int p = 0; p < n; p++) {
        double rho = 1.0 + perturb * orc_uniform(seed, 63, (uint64_t)p);
        double *q = o->g + 12 * (size_t)p;
        q[0] = rho;
        q[1] = kind[p] == 1 ? 0.0 : o->u0;
        q[2] = 0.0;
        for (int i = 0; i < 9; i++) q[3 + i] = 0.0;
    }
    /* make the initial state consistent across the interfaces */
    if (!o->periodic0) apply_outer_bc(o);
    for (int c = 1; c < L; c++) {
        snapshot(o, c - 1, o->lv[c - 1].snapA);
        snapshot(o, c - 1, o->lv[c - 1].snapB);
        prolong(o, c - 1, 0.0);
    }
    for (int c = L - 2; c >= 0; c--) restrict_level(o, c);
    if (n > 0) {
        ring_interp(o, o->Q0);
        ring_interp(o, o->Q1);
        ring_set(o, 0.0);
    }
    return o;
}

/* ------------------------------------------------------------ queries ---- */
/* Host threads the node loops use (1 in the serial build). */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Strength of the odd-even filter of the mesh state (fv_filter; 0 = off). */
void orc_set_fv_filter(orc *o, double sigma) { o->fv_filter = sigma; }

/* Test hook: apply the level-0 outer conditions to the current state. */
void orc_apply_outer_bc(orc *o) { apply_outer_bc(o); }


int orc_n_sub(const orc *o) { return o->n_sub; }
double orc_tau(const orc *o, int c) { return c < 0 ? o->tau_u : o->lv[c].tau; }
long orc_step_count(const orc *o) { return o->step; }
int orc_n_forces(const orc *o) { return o->nf; }

void orc_forces(const orc *o, double *cd, double *cl)
{
    memcpy(cd, o->cd, (size_t)o->nf * sizeof(double));
    memcpy(cl, o->cl, (size_t)o->nf * sizeof(double));
}

/* Density and velocity of grid `grid` (-1: mesh, else level index); NaN on
 * nodes that are not computed (the hole and its interpolation nodes). */
int orc_fields(const orc *o, int grid, double *rho, double *ux, double *uy)
{
    if (grid == -1) {
        for (int p = 0; p < o->n; p++) {
            rho[p] = o->g[12 * (size_t)p];
            ux[p] = o->g[12 * (size_t)p + 1];
            uy[p] = o->g[12 * (size_t)p + 2];
        }
        return o->n;
    }
    if (grid < 0 || grid >= o->L) return -1;
    const olevel *l = &o->lv[grid];
    size_t nn = (size_t)l->nx * l->ny;
    for (size_t p = 0; p < nn; p++) {
        if (l->type[p] == T_HOLE || l->type[p] == T_INTERP) { rho[p] = ux[p] = uy[p] = NAN; continue; }
        orc_moments(l->f + 9 * p, &rho[p], &ux[p], &uy[p]);
    }
    return (int)nn;
}

/* Raw populations of a grid (-1: mesh) into out (node-major, 9 per node). */
int orc_populations(const orc *o, int grid, double *out)
{
    if (grid == -1) {
        for (int p = 0; p < o->n; p++) from_q(o->g + 12 * (size_t)p, 1.0, out + 9 * (size_t)p);
        return o->n;
    }
    const olevel *l = &o->lv[grid];
    size_t nn = (size_t)l->nx * l->ny;
    memcpy(out, l->f, nn * 9 * sizeof(double));
    return (int)nn;
}

/* Overwrite the populations of a grid (-1: mesh) from node-major `f`
 * (test hook for initial conditions other than the uniform stream). */
int orc_set_populations(orc *o, int grid, const double *f)
{
    if (grid == -1) {
        for (int p = 0; p < o->n; p++) state_q(f + 9 * (size_t)p, o->g + 12 * (size_t)p);
        return o->n;
    }
    if (grid < 0 || grid >= o->L) return -1;
    olevel *l = &o->lv[grid];
    size_t nn = (size_t)l->nx * l->ny;
    memcpy(l->f, f, nn * 9 * sizeof(double));
    return (int)nn;
}

/* Set-up tables for comparison with other implementations.  Returns the
 * number of values (call with out == NULL to size). */
long orc_table(const orc *o, const char *name, double *out)
{
    long n = -1;
#define EMIT(count, expr) do { n = (long)(count); if (out) for (long k_ = 0; k_ < n; k_++) out[k_] = (double)(expr); } while (0)
    if (!strcmp(name, "rowptr")) EMIT(o->n + 1, o->rowptr[k_]);
    else if (!strcmp(name, "col")) EMIT(o->nnz, o->col[k_]);
    else if (!strcmp(name, "sx")) EMIT(o->nnz, o->sx[k_]);
    else if (!strcmp(name, "sy")) EMIT(o->nnz, o->sy[k_]);
    else if (!strcmp(name, "cc")) EMIT(o->nnz, o->cc[k_]);
    else if (!strcmp(name, "area")) EMIT(o->n, o->area[k_]);
    else if (!strcmp(name, "xy")) EMIT(2 * o->n, o->xy[k_]);
    else if (!strcmp(name, "is_node")) EMIT(o->n_is, o->is_node[k_]);
    else if (!strcmp(name, "is_don")) EMIT(6 * o->n_is, o->is_don[k_]);
    else if (!strcmp(name, "is_w")) EMIT(6 * o->n_is, o->is_w[k_]);
    else if (!strcmp(name, "ring")) EMIT(o->n_ring, o->ring[k_]);
    else if (!strcmp(name, "ring_don")) EMIT(9 * o->n_ring, o->ring_don[k_]);
    else if (!strcmp(name, "ring_w")) EMIT(9 * o->n_ring, o->ring_w[k_]);
    else if (!strcmp(name, "wall_edges")) EMIT(2 * o->n_wedge, (k_ % 2) ? o->web[k_ / 2] : o->wea[k_ / 2]);
    else if (!strncmp(name, "type", 4)) {
        int c = atoi(name + 4);
        if (c >= 0 && c < o->L) EMIT((long)o->lv[c].nx * o->lv[c].ny, o->lv[c].type[k_]);
    }
#undef EMIT
    return n;
}
