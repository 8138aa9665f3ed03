// Discrete adjoint kernels of the HLBM step (FP64): the Eq. 3 sub-step with
// the wall rule and the Eq. 10-11 wall-force functional (below), the lattice
// side of a coupled step (collision, outer conditions, Eq. 4 + 8 and Eq. 9
// coupling), the refinement interface (band snapshot, prolongation,
// restriction), and the geometry derivatives (Eq. 3 operators, wall normals,
// Eq. 8 and Eq. 9 weights).  The host schedule that runs them in reverse is
// in api.cu (hlbm_adjoint, hlbm_fv_adjoint).
//
// The sub-step maps the mesh state of every node, stored as q = (rho - 1, u_x,
// u_y, f^neq_3..8) (f^neq_0..2 follow from the zero mass and momentum of
// f^neq), to the next one; row P of the map reads P and its neighbours P_k:
//   acc_i = sum_k (c_i . s_k dt) [f^eq_i(P_k) - f^eq_i(P) + f^neq_i(P_k) - f^neq_i(P)]
//           - sum_k (dt / tau_u) C_Pk f^neq_i(P_k) - (dt / tau_u) C_PP f^neq_i(P)
//   rho' = rho + sum_i acc_i,  rho' u' = rho u + sum_i c_i acc_i,
//   f^neq_i' = f^neq_i + acc_i - [f^eq_i(rho', u') - f^eq_i(rho, u)]
// (the self term of the streaming sum vanishes because sum_k s_k = 0 over a
// closed control volume; C_PP = 11/18 on every node), then u' = 0 on wall
// nodes and, except after the last sub-step of a finest step, the interface
// rows take Eq. 5-7 values that do not depend on the mesh state.
//
// The transpose of one sub-step takes two launches.  Per row P (k_adj_rows):
// the cotangent of P's output through the node-local update gives mu =
// dJ/d(acc) and, with the terms of acc that read P itself, P's own share
// sig; both are forward-mode dual numbers over nine lanes.  Per node Q
// (k_adj_gather): sig(Q) plus, over the rows that have Q as a neighbour, mu
// contracted with the derivative of that neighbour term (Q's node-local
// Jacobian, evaluated once), and the entry's coefficient gradient.  Every
// output has one writer, so the result is deterministic (no atomics).
#include <cuda_runtime.h>

#include <algorithm>

#include "hlbm_device.h"

namespace hlbm {
namespace {

constexpr int kLanes = 9;  // derivative lanes: the nine state (or increment) components

struct Dual {
    double v;
    double d[kLanes];
};

__device__ __forceinline__ Dual cst(double v)
{
    Dual r;
    r.v = v;
#pragma unroll
    for (int l = 0; l < kLanes; l++) r.d[l] = 0.0;
    return r;
}
__device__ __forceinline__ Dual seeded(double v, int lane)
{
    Dual r = cst(v);
    if (lane >= 0) r.d[lane] = 1.0;
    return r;
}
__device__ __forceinline__ Dual operator+(const Dual &a, const Dual &b)
{
    Dual r;
    r.v = a.v + b.v;
#pragma unroll
    for (int l = 0; l < kLanes; l++) r.d[l] = a.d[l] + b.d[l];
    return r;
}
__device__ __forceinline__ Dual operator-(const Dual &a, const Dual &b)
{
    Dual r;
    r.v = a.v - b.v;
#pragma unroll
    for (int l = 0; l < kLanes; l++) r.d[l] = a.d[l] - b.d[l];
    return r;
}
__device__ __forceinline__ Dual operator*(const Dual &a, const Dual &b)
{
    Dual r;
    r.v = a.v * b.v;
#pragma unroll
    for (int l = 0; l < kLanes; l++) r.d[l] = a.d[l] * b.v + a.v * b.d[l];
    return r;
}
__device__ __forceinline__ Dual operator*(double a, const Dual &b)
{
    Dual r;
    r.v = a * b.v;
#pragma unroll
    for (int l = 0; l < kLanes; l++) r.d[l] = a * b.d[l];
    return r;
}
__device__ __forceinline__ Dual operator/(const Dual &a, const Dual &b)
{
    Dual r;
    const double ib = 1.0 / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int l = 0; l < kLanes; l++) r.d[l] = (a.d[l] - r.v * b.d[l]) * ib;
    return r;
}

// D2Q9: (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
__constant__ int kCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__constant__ double kW[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

// Eq. 2: f^eq_i(rho, u) = w_i rho [1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u]
__device__ __forceinline__ Dual feq(int i, const Dual &rho, const Dual &ux, const Dual &uy)
{
    const Dual cu = double(kCx[i]) * ux + double(kCy[i]) * uy;
    const Dual uu = ux * ux + uy * uy;
    return kW[i] * (rho * (cst(1.0) + 3.0 * cu + 4.5 * (cu * cu) - 1.5 * uu));
}

// f^neq_0..2 from the stored f^neq_3..8: zero mass and momentum
__device__ __forceinline__ void complete(Dual n[9])
{
    n[1] = n[3] - n[5] + n[6] + n[7] - n[8];
    n[2] = n[4] - n[5] - n[6] + n[7] + n[8];
    n[0] = cst(0.0) - (n[1] + n[2] + n[3] + n[4] + n[5] + n[6] + n[7] + n[8]);
}

// state of node k as duals, seeded on lanes 0..8 when seed is set
__device__ __forceinline__ void load(const double *g, int Np, int k, bool seed, Dual &rho, Dual &ux, Dual &uy,
                                     Dual n[9])
{
    rho = seeded(1.0 + g[k], seed ? 0 : -1);  // lane 0: rho - 1
    ux = seeded(g[size_t(Np) + k], seed ? 1 : -1);
    uy = seeded(g[size_t(2) * Np + k], seed ? 2 : -1);
#pragma unroll
    for (int i = 3; i < 9; i++) n[i] = seeded(g[size_t(i) * Np + k], seed ? i : -1);
    complete(n);
}

__device__ __forceinline__ double feqd(int i, double rho, double ux, double uy)
{
    const double cu = kCx[i] * ux + kCy[i] * uy;
    return kW[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy));
}

// Forward data of row P in double: its state, f^eq(P), the completed f^neq(P),
// the increments acc_i and the sums (Sa, Sb) of its entries' (a, b).
__device__ void row_forward(const double *g, int Np, int P, const int *rp, const int *rcol, const double *rcoef,
                            double csP, double &r1, double &ux, double &uy, double nP[9], double eqP[9],
                            double acc[9], double &Sa, double &Sb)
{
    r1 = g[P];
    ux = g[size_t(Np) + P];
    uy = g[size_t(2) * Np + P];
    for (int i = 3; i < 9; i++) nP[i] = g[size_t(i) * Np + P];
    nP[1] = nP[3] - nP[5] + nP[6] + nP[7] - nP[8];
    nP[2] = nP[4] - nP[5] - nP[6] + nP[7] + nP[8];
    nP[0] = -(nP[1] + nP[2] + nP[3] + nP[4] + nP[5] + nP[6] + nP[7] + nP[8]);
    for (int i = 0; i < 9; i++) {
        eqP[i] = feqd(i, 1.0 + r1, ux, uy);
        acc[i] = -csP * nP[i];
    }
    Sa = Sb = 0.0;
    for (int e = rp[P]; e < rp[P + 1]; e++) {
        const int k = rcol[e];
        const double a = rcoef[3 * size_t(e)], b = rcoef[3 * size_t(e) + 1], cs = rcoef[3 * size_t(e) + 2];
        Sa += a;
        Sb += b;
        const double rk = 1.0 + g[k], ukx = g[size_t(Np) + k], uky = g[size_t(2) * Np + k];
        double nk[9];
        for (int i = 3; i < 9; i++) nk[i] = g[size_t(i) * Np + k];
        nk[1] = nk[3] - nk[5] + nk[6] + nk[7] - nk[8];
        nk[2] = nk[4] - nk[5] - nk[6] + nk[7] + nk[8];
        nk[0] = -(nk[1] + nk[2] + nk[3] + nk[4] + nk[5] + nk[6] + nk[7] + nk[8]);
        for (int i = 0; i < 9; i++)
            acc[i] += (kCx[i] * a + kCy[i] * b) * (feqd(i, rk, ukx, uky) - eqP[i] + nk[i] - nP[i]) - cs * nk[i];
    }
}

// The update of row P from its increments (see the file comment).
__device__ void epilogue(const Dual &rP, const Dual &uPx, const Dual &uPy, const Dual nP[9], const Dual eqP[9],
                         const Dual acc[9], bool wall, Dual out[9])
{
    Dual drho = cst(0.0), djx = cst(0.0), djy = cst(0.0);
#pragma unroll
    for (int i = 0; i < 9; i++) {
        drho = drho + acc[i];
        djx = djx + double(kCx[i]) * acc[i];
        djy = djy + double(kCy[i]) * acc[i];
    }
    const Dual rho2 = rP + drho;
    const Dual ux2 = uPx + (djx - drho * uPx) / rho2, uy2 = uPy + (djy - drho * uPy) / rho2;
    out[0] = rho2 - cst(1.0);
    out[1] = wall ? cst(0.0) : ux2;
    out[2] = wall ? cst(0.0) : uy2;
#pragma unroll
    for (int i = 3; i < 9; i++) out[i] = nP[i] + acc[i] - (feq(i, rho2, ux2, uy2) - eqP[i]);
}

// Eq. 10-11 traction of wall edge (a, b) (normal times length wn, into the
// fluid), contracted with (wd, wl) / q; derivatives with respect to node
// `seed_node`'s state.
__device__ Dual edge_functional(const double *g, int Np, int a, int b, double nx, double ny, int seed_node, double wd,
                                double wl, double inv_q)
{
    Dual p = cst(0.0), pxx = cst(0.0), pxy = cst(0.0), pyy = cst(0.0);
    for (int s = 0; s < 2; s++) {
        const int k = s ? b : a;
        Dual r, ux, uy, n[9];
        load(g, Np, k, k == seed_node, r, ux, uy, n);
        p = p + (0.5 / 3.0) * r;
#pragma unroll
        for (int i = 0; i < 9; i++) {
            pxx = pxx + double(0.5 * kCx[i] * kCx[i]) * n[i];
            pxy = pxy + double(0.5 * kCx[i] * kCy[i]) * n[i];
            pyy = pyy + double(0.5 * kCy[i] * kCy[i]) * n[i];
        }
    }
    const Dual pm = p - cst(1.0 / 3.0);
    const Dual fx = cst(0.0) - nx * pm - (nx * pxx + ny * pxy);
    const Dual fy = cst(0.0) - ny * pm - (nx * pxy + ny * pyy);
    return inv_q * (wd * fx + wl * fy);
}

// J = sum over wall edges, one block, fixed order (deterministic)
__global__ void __launch_bounds__(256) k_adj_value(const double *g, int Np, const int *wea, const int *web,
                                                   const double *wn, int n_edges, double wd, double wl, double inv_q,
                                                   double *J)
{
    __shared__ double part[256];
    double s = 0.0;
    for (int e = threadIdx.x; e < n_edges; e += blockDim.x)
        s += edge_functional(g, Np, wea[e], web[e], wn[2 * e], wn[2 * e + 1], -1, wd, wl, inv_q).v;
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *J = part[0];
}

// cotangent of the final state: dJ/dq on wall nodes (through their edges),
// zero elsewhere; added to lam when add is set
__global__ void k_adj_terminal(const double *g, int Np, int n, const int *wptr, const int *wedge, const int *wea,
                               const int *web, const double *wn, double wd, double wl, double inv_q, int add,
                               double *lam)
{
    const int Q = blockIdx.x * blockDim.x + threadIdx.x;
    if (Q >= n) return;
    double d[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = wptr[Q]; t < wptr[Q + 1]; t++) {  // the wall edges of node Q (none off the wall)
        const int e = wedge[t];
        const Dual f = edge_functional(g, Np, wea[e], web[e], wn[2 * e], wn[2 * e + 1], Q, wd, wl, inv_q);
#pragma unroll
        for (int l = 0; l < 9; l++) d[l] += f.d[l];
    }
#pragma unroll
    for (int l = 0; l < 9; l++) lam[size_t(l) * Np + Q] = (add ? lam[size_t(l) * Np + Q] : 0.0) + d[l];
}

// Reverse sub-step, part 1 (one thread per row P).  With lam the cotangent
// of row P's output: mu_i = dJ/d acc_i (through the update alone) and
// sig = dJ/d(P's own state) through the update and through the terms of acc
// that read P (-S_i (f^eq_i(P) + f^neq_i(P)) - C_PP dt/tau f^neq_i(P), S_i =
// c_i . sum_k (a_k, b_k)).  E_i = f^eq_i(P) + f^neq_i(P) is kept for part 2.
// Interface rows overwritten after this sub-step (star) read nothing.
__global__ void __launch_bounds__(128) k_adj_rows(const double *g, int Np, int n, const int *rp, const int *rcol,
                                                  const double *rcoef, double csP, int n_wall, int ring_start,
                                                  int star, const double *lam_in, double *mu, double *sig, double *E)
{
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= n) return;
    double lam[9];
    bool any = false;
    for (int o = 0; o < 9; o++) {
        lam[o] = lam_in[size_t(o) * Np + P];
        any |= lam[o] != 0.0;
    }
    if (!any || (star && P >= ring_start)) {
        for (int l = 0; l < 9; l++) {
            mu[size_t(l) * Np + P] = 0.0;
            sig[size_t(l) * Np + P] = 0.0;
            E[size_t(l) * Np + P] = 0.0;
        }
        return;
    }
    const bool wall = P < n_wall;
    double r1, ux, uy, nP[9], eqP[9], acc[9], Sa, Sb;
    row_forward(g, Np, P, rp, rcol, rcoef, csP, r1, ux, uy, nP, eqP, acc, Sa, Sb);
    for (int i = 0; i < 9; i++) E[size_t(i) * Np + P] = eqP[i] + nP[i];
    {  // mu: seeds on the increments
        Dual nPd[9], eqd[9], accd[9], out[9];
        for (int i = 0; i < 9; i++) {
            nPd[i] = cst(nP[i]);
            eqd[i] = cst(eqP[i]);
            accd[i] = seeded(acc[i], i);
        }
        epilogue(cst(1.0 + r1), cst(ux), cst(uy), nPd, eqd, accd, wall, out);
        for (int l = 0; l < 9; l++) {
            double m = 0.0;
            for (int o = 0; o < 9; o++) m += lam[o] * out[o].d[l];
            mu[size_t(l) * Np + P] = m;
        }
    }
    {  // sig: seeds on P's state
        Dual rPd, uxd, uyd, nPd[9], eqd[9], accd[9], out[9];
        load(g, Np, P, true, rPd, uxd, uyd, nPd);
        for (int i = 0; i < 9; i++) {
            eqd[i] = feq(i, rPd, uxd, uyd);
            const double Si = kCx[i] * Sa + kCy[i] * Sb;
            const Dual X = cst(0.0) - Si * (eqd[i] + nPd[i]) - csP * nPd[i];
            accd[i] = cst(acc[i]) + (X - cst(X.v));
        }
        epilogue(rPd, uxd, uyd, nPd, eqd, accd, wall, out);
        for (int l = 0; l < 9; l++) {
            double m = 0.0;
            for (int o = 0; o < 9; o++) m += lam[o] * out[o].d[l];
            sig[size_t(l) * Np + P] = m;
        }
    }
}

// Reverse sub-step, part 2 (one thread per node Q): lam_out(Q) = sig(Q) plus,
// over the rows P having Q as neighbour entry e = (a, b, cs),
//   sum_i mu_i(P) [(c_i . (a, b)) d(f^eq_i(Q) + f^neq_i(Q)) - cs d f^neq_i(Q)],
// and the entry's gradient dJ/d(a, b, cs) = sum_i mu_i(P) (c_i (F_i(Q) - E_i(P)),
// -f^neq_i(Q)), added (times dt, dt, dt/tau: the unscaled s_x, s_y, C) to
// gcoef [nnz][3] in plan order.  One writer per output: deterministic.
__global__ void __launch_bounds__(128) k_adj_gather(const double *g, int Np, int n, const int *rp,
                                                    const double *rcoef, const int *rcsr, const int *tp,
                                                    const int *trow, const int *tpos, int ring_start, int star,
                                                    double dt, double dt_tau, const double *mu, const double *sig,
                                                    const double *E, double *lam_out, double *gcoef)
{
    const int Q = blockIdx.x * blockDim.x + threadIdx.x;
    if (Q >= n) return;
    double d[9];
    for (int l = 0; l < 9; l++) d[l] = sig[size_t(l) * Np + Q];
    Dual rQ, uxQ, uyQ, nQ[9], F[9];
    load(g, Np, Q, true, rQ, uxQ, uyQ, nQ);
    for (int i = 0; i < 9; i++) F[i] = feq(i, rQ, uxQ, uyQ) + nQ[i];
    for (int t = tp[Q]; t < tp[Q + 1]; t++) {
        const int P = trow[t], pos = tpos[t];
        if (pos < 0 || (star && P >= ring_start)) continue;
        double m[9];
        bool any = false;
        for (int i = 0; i < 9; i++) {
            m[i] = mu[size_t(i) * Np + P];
            any |= m[i] != 0.0;
        }
        if (!any) continue;
        const int e = rp[P] + pos;
        const double a = rcoef[3 * size_t(e)], b = rcoef[3 * size_t(e) + 1], cs = rcoef[3 * size_t(e) + 2];
        double ga = 0.0, gb = 0.0, gcs = 0.0;
        for (int i = 0; i < 9; i++) {
            const double S = kCx[i] * a + kCy[i] * b;
            for (int l = 0; l < 9; l++) d[l] += m[i] * (S * F[i].d[l] - cs * nQ[i].d[l]);
            const double D = F[i].v - E[size_t(i) * Np + P];
            ga += m[i] * kCx[i] * D;
            gb += m[i] * kCy[i] * D;
            gcs -= m[i] * nQ[i].v;
        }
        double *gc = gcoef + 3 * size_t(rcsr[e]);
        gc[0] += dt * ga;
        gc[1] += dt * gb;
        gc[2] += dt_tau * gcs;
    }
    for (int l = 0; l < 9; l++) lam_out[size_t(l) * Np + Q] = d[l];
}

// dJ / d(populations) of the window's initial state, input node order:
// g_i = f^eq_i(rho, u) + f^neq_i maps to q by rho = sum g, rho u = sum c g,
// f^neq_i = g_i - f^eq_i(rho, u).
__global__ void k_adj_populations(const double *g, int Np, int n, const int *perm, const double *lam, double *grad)
{
    const int Q = blockIdx.x * blockDim.x + threadIdx.x;
    if (Q >= n) return;
    Dual r, ux, uy, nq[9];
    load(g, Np, Q, false, r, ux, uy, nq);
    Dual f[9];
#pragma unroll
    for (int i = 0; i < 9; i++) f[i] = seeded(feq(i, r, ux, uy).v + nq[i].v, i);
    Dual rho = cst(0.0), jx = cst(0.0), jy = cst(0.0);
#pragma unroll
    for (int i = 0; i < 9; i++) {
        rho = rho + f[i];
        jx = jx + double(kCx[i]) * f[i];
        jy = jy + double(kCy[i]) * f[i];
    }
    const Dual vx = jx / rho, vy = jy / rho;
    Dual q[9];
    q[0] = rho - cst(1.0);
    q[1] = vx;
    q[2] = vy;
#pragma unroll
    for (int i = 3; i < 9; i++) q[i] = f[i] - feq(i, rho, vx, vy);
    const int p = perm[Q];
#pragma unroll
    for (int l = 0; l < 9; l++) {
        double s = 0.0;
#pragma unroll
        for (int o = 0; o < 9; o++) s += lam[size_t(o) * Np + Q] * q[o].d[l];
        grad[9 * size_t(p) + l] = s;
    }
}

// ------------------------------------------------ geometry (shape) part ----
// The Eq. 3 entries of row P are U_Pk / A_P: U sums, per triangle (P, A, B)
// counter-clockwise (edge vectors a = x_A - x_P, b = x_B - x_P),
//   s_PP: -5/24 perp(b - a),  s_PA: -1/24 perp(4b - 3a),  s_PB: -1/24 perp(3b - 4a),
//   C_PP: 11/54 |T|,  C_PA, C_PB: 7/108 |T|,   A_P: |T| / 3,
// and per boundary edge a -> b: s_aa, s_bb: -3/8 perp(x_b - x_a), s_ab, s_ba:
// -1/8 perp(x_b - x_a), with perp(d) = (d_y, -d_x).  With G_e = dJ/d(entry e)
// the chain rule gives dJ/dU_e = G_e / A_P and dJ/dA_P = -sum_e G_e . c_e / A_P.
// The wall force reads the edge normals n_e = (-d_y, d_x), d = x_b - x_a.

// -sum_e G_e . c_e / A_P per row
__global__ void k_adj_abar(const int *prow, const double *pcoef, const double *gc, const double *parea, int n,
                           double *abar)
{
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= n) return;
    double s = 0.0;
    for (int e = prow[P]; e < prow[P + 1]; e++)
        for (int c = 0; c < 3; c++) s += gc[3 * size_t(e) + c] * pcoef[3 * size_t(e) + c];
    abar[P] = -s / parea[P];
}

// dJ/dn_e of each wall edge: the traction -(p - p0) n - Pi^neq n of the final
// state contracted with (wd, wl) / q
__global__ void k_adj_wall_normal(const double *g, int Np, const int *inv, const int *iwea, const int *iweb,
                                  int n_edges, double wd, double wl, double inv_q, int add, double *h)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_edges) return;
    double p = 0.0, pxx = 0.0, pxy = 0.0, pyy = 0.0;
    for (int s = 0; s < 2; s++) {
        const int k = inv[s ? iweb[e] : iwea[e]];
        Dual r, ux, uy, nq[9];
        load(g, Np, k, false, r, ux, uy, nq);
        p += (0.5 / 3.0) * r.v;
        for (int i = 0; i < 9; i++) {
            pxx += 0.5 * kCx[i] * kCx[i] * nq[i].v;
            pxy += 0.5 * kCx[i] * kCy[i] * nq[i].v;
            pyy += 0.5 * kCy[i] * kCy[i] * nq[i].v;
        }
    }
    const double pm = p - 1.0 / 3.0;
    // J_e = inv_q [wd (-pm n_x - pxx n_x - pxy n_y) + wl (-pm n_y - pxy n_x - pyy n_y)]
    h[2 * e] = (add ? h[2 * e] : 0.0) + inv_q * (wd * (-pm - pxx) - wl * pxy);
    h[2 * e + 1] = (add ? h[2 * e + 1] : 0.0) + inv_q * (-wd * pxy + wl * (-pm - pyy));
}

__device__ __forceinline__ int find_entry(const int *prow, const int *pcol, int row, int c)
{
    int lo = prow[row], hi = prow[row + 1];
    const int end = hi;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pcol[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    // rows hold every vertex of their triangles; -1 (no term) otherwise
    return lo < end && pcol[lo] == c ? lo : -1;
}

__device__ __forceinline__ double gget(const double *gc, int e, int c) { return e < 0 ? 0.0 : gc[3 * size_t(e) + c]; }

// dJ/dx of node X (posed frame), gathered over its triangles, boundary edges
// and wall edges; then the input frame (x_posed = p + R(-alpha)(x - p)).
__global__ void k_adj_shape(const AdjTables A, int n, const double *gc, const double *abar, const double *h,
                            double ca, double sa, double *gpos, double *grad_xy)
{
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    if (X >= n) return;
    double gx = 0.0, gy = 0.0;
    const double *xy = A.pxy;
    for (int j = A.ntp[X]; j < A.ntp[X + 1]; j++) {
        const int t = A.ntl[j];
        const int v[3] = {A.ptri[3 * t], A.ptri[3 * t + 1], A.ptri[3 * t + 2]};
        // d|T| / d(vertex k): 1/2 (y_{k+1} - y_{k+2}, x_{k+2} - x_{k+1})
        int kx = 0;
        for (int k = 0; k < 3; k++)
            if (v[k] == X) kx = k;
        const int k1 = v[(kx + 1) % 3], k2 = v[(kx + 2) % 3];
        const double dax = 0.5 * (xy[2 * k1 + 1] - xy[2 * k2 + 1]), day = 0.5 * (xy[2 * k2] - xy[2 * k1]);
        for (int a = 0; a < 3; a++) {
            const int ip = v[a], ia = v[(a + 1) % 3], ib = v[(a + 2) % 3];
            const int ePP = find_entry(A.prow, A.pcol, ip, ip), ePA = find_entry(A.prow, A.pcol, ip, ia),
                      ePB = find_entry(A.prow, A.pcol, ip, ib);
            const double iA = 1.0 / A.parea[ip];
            // dJ/dU of the streaming entries, w = G / A_P, and d/d(d) of -k perp(d).w = k (w_y, -w_x)
            const double wPx = gget(gc, ePP, 0) * iA, wPy = gget(gc, ePP, 1) * iA;
            const double wAx = gget(gc, ePA, 0) * iA, wAy = gget(gc, ePA, 1) * iA;
            const double wBx = gget(gc, ePB, 0) * iA, wBy = gget(gc, ePB, 1) * iA;
            // d = b - a (5/24), 4b - 3a (1/24, entry A), 3b - 4a (1/24, entry B)
            const double gPx = (5.0 / 24.0) * wPy, gPy = -(5.0 / 24.0) * wPx;
            const double gAx = (1.0 / 24.0) * wAy, gAy = -(1.0 / 24.0) * wAx;
            const double gBx = (1.0 / 24.0) * wBy, gBy = -(1.0 / 24.0) * wBx;
            const double da_x = -gPx - 3.0 * gAx - 4.0 * gBx, da_y = -gPy - 3.0 * gAy - 4.0 * gBy;  // d/da
            const double db_x = gPx + 4.0 * gAx + 3.0 * gBx, db_y = gPy + 4.0 * gAy + 3.0 * gBy;    // d/db
            if (X == ia) { gx += da_x; gy += da_y; }
            if (X == ib) { gx += db_x; gy += db_y; }
            if (X == ip) { gx -= da_x + db_x; gy -= da_y + db_y; }
            // collision entries and the control-volume area, both multiples of |T|
            const double kap = (11.0 / 54.0) * gget(gc, ePP, 2) * iA +
                               (7.0 / 108.0) * (gget(gc, ePA, 2) + gget(gc, ePB, 2)) * iA + abar[ip] / 3.0;
            gx += kap * dax;
            gy += kap * day;
        }
    }
    for (int j = A.bptr[X]; j < A.bptr[X + 1]; j++) {
        const int b = A.blist[j], ea = A.bed[2 * b], eb = A.bed[2 * b + 1];
        double sx_ = 0.0, sy_ = 0.0;  // sum of k (w_y, -w_x) over the four half-edge terms
        const int e1 = find_entry(A.prow, A.pcol, ea, ea), e2 = find_entry(A.prow, A.pcol, ea, eb);
        const int e3 = find_entry(A.prow, A.pcol, eb, eb), e4 = find_entry(A.prow, A.pcol, eb, ea);
        const double ia_ = 1.0 / A.parea[ea], ib_ = 1.0 / A.parea[eb];
        const double ks[4] = {0.375 * ia_, 0.125 * ia_, 0.375 * ib_, 0.125 * ib_};
        const int es[4] = {e1, e2, e3, e4};
        for (int q = 0; q < 4; q++) {
            sx_ += ks[q] * gget(gc, es[q], 1);
            sy_ -= ks[q] * gget(gc, es[q], 0);
        }
        if (X == eb) { gx += sx_; gy += sy_; }
        if (X == ea) { gx -= sx_; gy -= sy_; }
    }
    for (int j = A.iwptr[X]; j < A.iwptr[X + 1]; j++) {
        const int e = A.iwlist[j];
        // n = (-d_y, d_x): dJ/dd = (h_y, -h_x)
        const double hx = h[2 * e], hy = h[2 * e + 1];
        if (X == A.iweb[e]) { gx += hy; gy -= hx; }
        if (X == A.iwea[e]) { gx -= hy; gy += hx; }
    }
    gpos[2 * X] = gx;
    gpos[2 * X + 1] = gy;
    if (!grad_xy) return;
    // input frame: x_posed - p = R (x - p), R = [[ca, sa], [-sa, ca]]; dJ/dx = R^T dJ/dx_posed
    grad_xy[2 * size_t(X)] = ca * gx - sa * gy;
    grad_xy[2 * size_t(X) + 1] = sa * gx + ca * gy;
}



// dJ/dalpha (per degree): sum_X dJ/dx_posed . d x_posed / d alpha, with
// x_posed - p = R(alpha) (x - p): d/dalpha = (-sa dx + ca dy, -sa dy - ca dx)
// for the input-frame offsets (dx, dy) = R^T (x_posed - p); one block, fixed order
__global__ void __launch_bounds__(256) k_adj_aoa(const double *xy, const double *gpos, int n, double ca, double sa,
                                                 double px, double py, double *out)
{
    __shared__ double part[256];
    double s = 0.0;
    for (int X = threadIdx.x; X < n; X += blockDim.x) {
        const double ox = xy[2 * X] - px, oy = xy[2 * X + 1] - py;
        const double dx = ca * ox - sa * oy, dy = sa * ox + ca * oy;
        s += gpos[2 * X] * (-sa * dx + ca * dy) + gpos[2 * X + 1] * (-sa * dy - ca * dx);
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0] * (3.14159265358979323846 / 180.0);
}

// ------------------------------------ lattice side of a coupled step ----
// Single-level configurations: the lattice (deviations d_i = f_i - w_i,
// FP64, AA layout) and the mesh exchange through Eq. 4 + 8 (hole nodes from
// mesh donors) and Eq. 9 (interface data Q from lattice donors).  Cotangents
// of the lattice live in the same slots as its state: lam[slot] = dJ/d(value
// in that slot).  Every forward kernel reads and writes whole slot sets of
// single nodes, so each adjoint below reads the cotangents of the slots a
// node wrote and writes (or adds) those of the slots it read, one writer per
// slot.  AA addressing, node n at parity p: state of direction i in plane i
// at n (p = 0) or plane opp(i) at n - c_i (p = 1); a collision writes
// direction i to plane opp(i) at n (p = 0) or plane i at n + c_i (p = 1).
__constant__ int kOpp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

__device__ __forceinline__ size_t lnode(int x, int y, int pitch) { return size_t(y + 1) * pitch + x + 1; }
template <int P> __device__ __forceinline__ size_t lst(int i, size_t n, int pitch, size_t stride)
{
    if (P == 0) return size_t(i) * stride + n;
    return size_t(kOpp[i]) * stride + n - kCx[i] - ptrdiff_t(kCy[i]) * pitch;
}
template <int P> __device__ __forceinline__ size_t lwr(int i, size_t n, int pitch, size_t stride)
{
    if (P == 0) return size_t(kOpp[i]) * stride + n;
    return size_t(i) * stride + n + kCx[i] + ptrdiff_t(kCy[i]) * pitch;
}

// populations of node n (slots at parity P) as duals seeded on lanes 0..8
template <int P>
__device__ __forceinline__ void lat_load(const double *f, size_t n, int pitch, size_t stride, Dual F[9], Dual &rho,
                                         Dual &ux, Dual &uy)
{
    rho = cst(0.0);
    Dual jx = cst(0.0), jy = cst(0.0);
#pragma unroll
    for (int i = 0; i < 9; i++) {
        F[i] = seeded(f[lst<P>(i, n, pitch, stride)] + kW[i], i);
        rho = rho + F[i];
        jx = jx + double(kCx[i]) * F[i];
        jy = jy + double(kCy[i]) * F[i];
    }
    ux = jx / rho;
    uy = jy / rho;
}

// Eq. 1 (BGK collision at parity P, every computed node): the state before the
// collision f, cotangents of the written slots -> those of the read slots
// (the same slot set, in place).
template <int P>
__global__ void __launch_bounds__(128) k_adj_collide(const double *f, int nx, int ny, int pitch, size_t stride,
                                                     double omega, const int *hx0, const int *hx1, double *lam)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    if (hx0 && x >= hx0[y] && x < hx1[y]) return;
    const size_t n = lnode(x, y, pitch);
    Dual F[9], rho, ux, uy;
    lat_load<P>(f, n, pitch, stride, F, rho, ux, uy);
    double lp[9];
#pragma unroll
    for (int i = 0; i < 9; i++) lp[i] = lam[lwr<P>(i, n, pitch, stride)];
    double d[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const Dual post = F[i] - omega * (F[i] - feq(i, rho, ux, uy));
#pragma unroll
        for (int l = 0; l < 9; l++) d[l] += lp[i] * post.d[l];
    }
#pragma unroll
    for (int l = 0; l < 9; l++) lam[lst<P>(l, n, pitch, stride)] = d[l];
}

// Outer conditions (level 0, parity P, after the collision): perimeter node
// (x, y) takes the state of interior node (clamp x, clamp y): inlet x = 0
// f^eq(rho, (u0, 0)) + f^neq, outlet x = nx - 1 f^eq(1, u) + f^neq, else a
// copy.  Part 1, per interior frame node T: add the perimeter nodes' share.
template <int P>
__global__ void __launch_bounds__(128) k_adj_bc_gather(const double *f, int nx, int ny, int pitch, size_t stride,
                                                       double u0, double *lam)
{
    const int X = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y + 1;
    if (X < 1 || X > nx - 2 || Y > ny - 2) return;
    if (X != 1 && X != nx - 2 && Y != 1 && Y != ny - 2) return;  // not on the inner frame
    const size_t nT = lnode(X, Y, pitch);
    Dual F[9], rho, ux, uy;
    lat_load<P>(f, nT, pitch, stride, F, rho, ux, uy);
    double d[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int xs[3] = {X, X == 1 ? 0 : -1, X == nx - 2 ? nx - 1 : -1};
    const int ys[3] = {Y, Y == 1 ? 0 : -1, Y == ny - 2 ? ny - 1 : -1};
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            const int x = xs[a], y = ys[b];
            if (x < 0 || y < 0 || (a == 0 && b == 0)) continue;
            const size_t np = lnode(x, y, pitch);
            for (int i = 0; i < 9; i++) {
                const double lp = lam[lst<P>(i, np, pitch, stride)];
                if (lp == 0.0) continue;
                Dual out;
                if (x == 0) out = feq(i, rho, cst(u0), cst(0.0)) + F[i] - feq(i, rho, ux, uy);
                else if (x == nx - 1) out = feq(i, cst(1.0), ux, uy) + F[i] - feq(i, rho, ux, uy);
                else out = F[i];
                for (int l = 0; l < 9; l++) d[l] += lp * out.d[l];
            }
        }
#pragma unroll
    for (int l = 0; l < 9; l++) lam[lst<P>(l, nT, pitch, stride)] += d[l];
}

// Part 2: the perimeter slots were overwritten: their cotangents end here.
template <int P>
__global__ void k_adj_bc_clear(int nx, int ny, int pitch, size_t stride, double *lam)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int nper = 2 * nx + 2 * (ny - 2);
    if (k >= nper) return;
    int x, y;
    if (k < nx) { x = k; y = 0; }
    else if (k < 2 * nx) { x = k - nx; y = ny - 1; }
    else if (k < 2 * nx + ny - 2) { x = 0; y = k - 2 * nx + 1; }
    else { x = nx - 1; y = k - 2 * nx - (ny - 2) + 1; }
    const size_t n = lnode(x, y, pitch);
#pragma unroll
    for (int i = 0; i < 9; i++) lam[lst<P>(i, n, pitch, stride)] = 0.0;
}

// Eq. 9 (interface data Q[12][n_ring] = sum_k w_rk (rho, u, f - f^eq) of
// lattice donor k at parity P): cotangents lamQ -> the donors' slots.  Per
// lattice node: the (ring node, donor position) pairs that read it,
// lent[lptr[node] .. lptr[node + 1]) as 9 r + k, node = y nx + x.
template <int P>
__global__ void __launch_bounds__(128) k_adj_ring_lattice(const double *f, int nx, int ny, int pitch, size_t stride,
                                                          const int *lptr, const int *lent, const double *ring_w,
                                                          const double *lamQ, int n_ring, double *lam)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const int node = y * nx + x;
    if (lptr[node] == lptr[node + 1]) return;
    const size_t n = lnode(x, y, pitch);
    Dual F[9], rho, ux, uy;
    lat_load<P>(f, n, pitch, stride, F, rho, ux, uy);
    Dual q[12];
    q[0] = rho;
    q[1] = ux;
    q[2] = uy;
#pragma unroll
    for (int i = 0; i < 9; i++) q[3 + i] = F[i] - feq(i, rho, ux, uy);
    double d[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = lptr[node]; t < lptr[node + 1]; t++) {
        const int r = lent[t] / 9;
        const double w = ring_w[lent[t]];
        for (int m = 0; m < 12; m++) {
            const double lq = w * lamQ[size_t(m) * n_ring + r];
#pragma unroll
            for (int l = 0; l < 9; l++) d[l] += lq * q[m].d[l];
        }
    }
#pragma unroll
    for (int l = 0; l < 9; l++) lam[lst<P>(l, n, pitch, stride)] += d[l];
}

// Eq. 4 + 8, part 1 (per structured interpolation node s at parity P): the
// node's written slots held f^eq(q) + scale4 f^neq(q) with q = sum_k w_sk q(mesh
// donor k) (mesh state g); their cotangents -> lamq[12][n_is], and end there.
template <int P>
__global__ void k_adj_hole_q(const double *g, int Np, const int *is_n, const int *is_don, const double *is_w,
                             int n_is, double scale4, int pitch, size_t stride, double *lam, double *lamq, double *lw6)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_is) return;
    double q[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 6; k++) {
        const int p = is_don[6 * s + k];
        const double w = is_w[6 * s + k];
        Dual r, ux, uy, nq[9];
        load(g, Np, p, false, r, ux, uy, nq);
        q[0] += w * r.v;
        q[1] += w * ux.v;
        q[2] += w * uy.v;
        for (int i = 0; i < 9; i++) q[3 + i] += w * nq[i].v;
    }
    const size_t n = size_t(is_n[s]);
    const Dual rho = seeded(q[0], 0), vx = seeded(q[1], 1), vy = seeded(q[2], 2);
    double lq[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 9; i++) {
        const size_t slot = lwr<P>(i, n, pitch, stride);
        const double lo = lam[slot];
        lam[slot] = 0.0;
        const Dual e = feq(i, rho, vx, vy);
        lq[0] += lo * e.d[0];
        lq[1] += lo * e.d[1];
        lq[2] += lo * e.d[2];
        lq[3 + i] = scale4 * lo;
    }
    for (int m = 0; m < 12; m++) lamq[size_t(m) * n_is + s] = lq[m];
    if (lw6)  // dJ/d(weight k) += q(donor k) . lamq
        for (int k = 0; k < 6; k++) {
            Dual r, ux, uy, nq[9];
            load(g, Np, is_don[6 * s + k], false, r, ux, uy, nq);
            double dot = lq[0] * r.v + lq[1] * ux.v + lq[2] * uy.v;
            for (int i = 0; i < 9; i++) dot += lq[3 + i] * nq[i].v;
            lw6[6 * s + k] += dot;
        }
}

// Part 2 (per mesh node): q(mesh node) = (1 + r1, u, f^neq_0..8), the last
// three of f^neq completed from the stored six; pairs (s, k) that read the
// node: hent[hptr[node] .. hptr[node + 1]) as 6 s + k.
__global__ void k_adj_hole_mesh(const double *g, int Np, int n, const int *hptr, const int *hent, const double *is_w,
                                const double *lamq, int n_is, double *lam_g)
{
    const int Q = blockIdx.x * blockDim.x + threadIdx.x;
    if (Q >= n || hptr[Q] == hptr[Q + 1]) return;
    Dual r, ux, uy, nq[9];
    load(g, Np, Q, true, r, ux, uy, nq);
    double d[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = hptr[Q]; t < hptr[Q + 1]; t++) {
        const int s = hent[t] / 6;
        const double w = is_w[hent[t]];
        for (int m = 0; m < 12; m++) {
            const double lq = w * lamq[size_t(m) * n_is + s];
            const Dual &qm = m == 0 ? r : (m == 1 ? ux : (m == 2 ? uy : nq[m - 3]));
            for (int l = 0; l < 9; l++) d[l] += lq * qm.d[l];
        }
    }
    for (int l = 0; l < 9; l++) lam_g[size_t(l) * Np + Q] += d[l];
}

// Interface rows of a mesh state set from Q = (1 - theta) Q0 + theta Q1
// (Eq. 5-7: rho - 1 = Q_rho - 1, u = Q_u, f^neq_i = scale5 Q_neq,i): their
// cotangents -> lamQ0 (weight wa), lamQ1 (weight wb), and end there.
__global__ void k_adj_ring_rows(double *lam_g, int Np, int ring_start, int n_ring, double scale5, double wa,
                                double wb, double *lamQ0, double *lamQ1)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_ring) return;
    const int R = ring_start + r;
    for (int k = 0; k < 9; k++) {
        const double l = lam_g[size_t(k) * Np + R];
        lam_g[size_t(k) * Np + R] = 0.0;
        const int m = k < 3 ? k : 3 + k;  // Q component of mesh plane k
        const double v = k < 3 ? l : scale5 * l;
        lamQ0[size_t(m) * n_ring + r] += wa * v;
        lamQ1[size_t(m) * n_ring + r] += wb * v;
    }
}

// dJ/d(lattice populations), grid order [ny nx][9], from the cotangents of
// the slots at parity P; hole nodes (not computed) get 0.
template <int P>
__global__ void k_adj_lattice_out(const double *lam, int nx, int ny, int pitch, size_t stride, const int *hx0,
                                  const int *hx1, double *grad)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const bool hole = hx0 && x >= hx0[y] && x < hx1[y];
    const size_t n = lnode(x, y, pitch);
    for (int i = 0; i < 9; i++)
        grad[9 * (size_t(y) * nx + x) + i] = hole ? 0.0 : lam[lst<P>(i, n, pitch, stride)];
}

// ------------------------------------------------ refinement interface ----
// q(node) = (rho, u, f - f^eq) of a lattice node as duals (lanes: populations)
template <int P>
__device__ __forceinline__ void lat_q(const double *f, size_t n, int pitch, size_t stride, Dual q[12])
{
    Dual F[9], rho, ux, uy;
    lat_load<P>(f, n, pitch, stride, F, rho, ux, uy);
    q[0] = rho;
    q[1] = ux;
    q[2] = uy;
#pragma unroll
    for (int i = 0; i < 9; i++) q[3 + i] = F[i] - feq(i, rho, ux, uy);
}

// Band snapshot of a parent level (band entry b <-> node (X, Y): the lines
// y = coy, coy + cmy for x in [cox - 1, cox + cmx] and x = cox, cox + cmx for
// y in [coy - 1, coy + cmy]; corner nodes are on two lines): cotangents of
// the snapshot [12][band_n] -> the node's slots at parity P.  One thread per
// node of the band's box.
template <int P>
__global__ void k_adj_snapshot(const double *f, int pitch, size_t stride, int cox, int coy, int cmx, int cmy,
                               const double *lamS, int band_n, double *lam)
{
    const int X = cox - 1 + int(blockIdx.x * blockDim.x + threadIdx.x), Y = coy - 1 + int(blockIdx.y);
    if (X > cox + cmx) return;
    const int w = cmx + 2, h = cmy + 2;
    int b[2], nb = 0;
    if (Y == coy) b[nb++] = X - (cox - 1);
    if (Y == coy + cmy) b[nb++] = w + X - (cox - 1);
    if (X == cox && nb < 2) b[nb++] = 2 * w + Y - (coy - 1);
    if (X == cox + cmx && nb < 2) b[nb++] = 2 * w + h + Y - (coy - 1);
    if (nb == 0) return;
    const size_t n = lnode(X, Y, pitch);
    Dual q[12];
    lat_q<P>(f, n, pitch, stride, q);
    double d[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = 0; t < nb; t++)
        for (int m = 0; m < 12; m++) {
            const double l = lamS[size_t(m) * band_n + b[t]];
#pragma unroll
            for (int k = 0; k < 9; k++) d[k] += l * q[m].d[k];
        }
#pragma unroll
    for (int k = 0; k < 9; k++) lam[lst<P>(k, n, pitch, stride)] += d[k];
}

// Prolongation, part 1 (per fine perimeter node k at parity P): its slots
// held f^eq(q) + scale f^neq(q) with q = sum_t w_t ((1 - theta) A_bt + theta B_bt)
// of the parent's band data; cotangents -> lamq[12][nper] (dJ/dq), and end.
template <int P>
__global__ void k_adj_prolong_q(int nx, int ny, int pitch, size_t stride, const double *A, const double *B,
                                int band_n, int cmx, int cmy, double theta, double scale, double *lam, double *lamq)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int nper = 2 * nx + 2 * (ny - 2);
    if (k >= nper) return;
    int i, j;
    if (k < nx) { i = k; j = 0; }
    else if (k < 2 * nx) { i = k - nx; j = ny - 1; }
    else if (k < 2 * nx + ny - 2) { i = 0; j = k - 2 * nx + 1; }
    else { i = nx - 1; j = k - 2 * nx - (ny - 2) + 1; }
    const int w = cmx + 2, h = cmy + 2;
    int base, pos, odd;
    if (j == 0 || j == ny - 1) {
        base = (j == 0) ? 0 : w;
        pos = (i >> 1) + 1;
        odd = i & 1;
    } else {
        base = 2 * w + ((i == 0) ? 0 : h);
        pos = (j >> 1) + 1;
        odd = j & 1;
    }
    double q[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int nd = odd ? 3 : 1;
    for (int t = 0; t < nd; t++) {
        const int b = base + pos + (odd ? t - 1 : 0);
        const double wk = odd ? (t == 0 ? -0.125 : (t == 1 ? 0.75 : 0.375)) : 1.0;
        for (int m = 0; m < 12; m++)
            q[m] += wk * ((1.0 - theta) * A[size_t(m) * band_n + b] + theta * B[size_t(m) * band_n + b]);
    }
    const Dual rho = seeded(q[0], 0), vx = seeded(q[1], 1), vy = seeded(q[2], 2);
    const size_t n = lnode(i, j, pitch);
    double lq[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int d = 0; d < 9; d++) {
        const size_t slot = lst<P>(d, n, pitch, stride);
        const double lo = lam[slot];
        lam[slot] = 0.0;
        const Dual e = feq(d, rho, vx, vy);
        lq[0] += lo * e.d[0];
        lq[1] += lo * e.d[1];
        lq[2] += lo * e.d[2];
        lq[3 + d] = scale * lo;
    }
    for (int m = 0; m < 12; m++) lamq[size_t(m) * nper + k] = lq[m];
}

// Part 2 (per band entry b): the (fine perimeter node, weight) pairs that read
// it, pk[pp[b] .. pp[b + 1]) with weights pw; adds to the band cotangents.
__global__ void k_adj_prolong_band(const int *pp, const int *pk, const double *pw, const double *lamq, int nper,
                                   int band_n, double theta, double *lamA, double *lamB)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= band_n) return;
    for (int m = 0; m < 12; m++) {
        double s = 0.0;
        for (int t = pp[b]; t < pp[b + 1]; t++) s += pw[t] * lamq[size_t(m) * nper + pk[t]];
        lamA[size_t(m) * band_n + b] += (1.0 - theta) * s;
        lamB[size_t(m) * band_n + b] += theta * s;
    }
}

// Restriction (coarse node (X, Y) one cell or more inside the child box, not
// in the hole, at parity PC, from fine node (2 (X - cox), 2 (Y - coy)) at
// parity PF: f^eq(q) + scale f^neq(q) of the fine q): cotangents of the
// coarse slots -> the fine node's slots; the coarse slots end there.
template <int PC, int PF>
__global__ void k_adj_restrict(const double *ff, int pitch_c, size_t stride_c, int pitch_f, size_t stride_f, int cox,
                               int coy, int cmx, int cmy, double scale, const int *hx0, const int *hx1, double *lamc,
                               double *lamf)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (a >= cmx - 1) return;
    const int X = cox + 1 + a, Y = coy + 1 + b;
    if (hx0 && X >= hx0[Y] && X < hx1[Y]) return;
    const size_t nc = lnode(X, Y, pitch_c), nf = lnode(2 * (X - cox), 2 * (Y - coy), pitch_f);
    Dual q[12];
    lat_q<PF>(ff, nf, pitch_f, stride_f, q);
    double d[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 9; i++) {
        const size_t slot = lst<PC>(i, nc, pitch_c, stride_c);
        const double lo = lamc[slot];
        lamc[slot] = 0.0;
        const Dual out = feq(i, q[0], q[1], q[2]) + scale * q[3 + i];
#pragma unroll
        for (int k = 0; k < 9; k++) d[k] += lo * out.d[k];
    }
#pragma unroll
    for (int k = 0; k < 9; k++) lamf[lst<PF>(k, nf, pitch_f, stride_f)] += d[k];
}

// ---------------------------------- geometry through the coupled step ----
// Eq. 9 weights: dJ/d(w_rk) += q(lattice donor k at parity P) . lamQ(r)
template <int P>
__global__ void k_adj_ring_weights(const double *f, int pitch, size_t stride, const int *ring_don,
                                   const double *lamQ, int n_ring, double *lw9)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_ring) return;
    for (int k = 0; k < 9; k++) {
        Dual q[12];
        lat_q<P>(f, size_t(ring_don[9 * r + k]), pitch, stride, q);
        double dot = 0.0;
        for (int m = 0; m < 12; m++) dot += q[m].v * lamQ[size_t(m) * n_ring + r];
        lw9[9 * r + k] += dot;
    }
}

// Eq. 8 weights reproduce {1, u, v, u^2, uv, v^2} at the interpolation node:
// sum_k w_k m_j(x_k - x_s) = [j == 0] (a scaling of u, v leaves w unchanged).
// With M_jk = m_j(d_k): dJ/dM = -z w^T, M^T z = dJ/dw, and dJ/dd_k =
// -w_k sum_j z_j grad m_j(d_k).  Part 1, per interpolation node: z.
__global__ void k_adj_eq8_solve(const int *isd_in, const double *is_xy, const double *pxy, const double *lw6, int n_is,
                                double *zs)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_is) return;
    double a[6][7];  // M^T | rhs
    for (int k = 0; k < 6; k++) {
        const int p = isd_in[6 * s + k];
        const double u = pxy[2 * p] - is_xy[2 * s], v = pxy[2 * p + 1] - is_xy[2 * s + 1];
        const double m[6] = {1.0, u, v, u * u, u * v, v * v};
        for (int j = 0; j < 6; j++) a[k][j] = m[j];  // row k of M^T = column k of M
        a[k][6] = lw6[6 * s + k];
    }
    for (int c = 0; c < 6; c++) {  // Gaussian elimination, partial pivoting
        int piv = c;
        for (int r = c + 1; r < 6; r++)
            if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
        if (piv != c)
            for (int j = 0; j < 7; j++) {
                const double t = a[c][j];
                a[c][j] = a[piv][j];
                a[piv][j] = t;
            }
        for (int r = 0; r < 6; r++) {
            if (r == c || a[c][c] == 0.0) continue;
            const double f = a[r][c] / a[c][c];
            for (int j = c; j < 7; j++) a[r][j] -= f * a[c][j];
        }
    }
    for (int j = 0; j < 6; j++) zs[6 * s + j] = a[j][j] == 0.0 ? 0.0 : a[j][6] / a[j][j];
}

// Part 2, per mesh node (device order Q, input node perm[Q]): over the
// (interpolation node s, donor position k) pairs that read it, add
// -w_sk sum_j z_sj grad m_j(x_Q - x_s) to its posed-frame gradient.
__global__ void k_adj_eq8_nodes(const int *hptr, const int *hent, const int *perm, const double *is_w,
                                const double *is_xy, const double *pxy, const double *zs, int n, double *gpos)
{
    const int Q = blockIdx.x * blockDim.x + threadIdx.x;
    if (Q >= n || hptr[Q] == hptr[Q + 1]) return;
    const int p = perm[Q];
    double gx = 0.0, gy = 0.0;
    for (int t = hptr[Q]; t < hptr[Q + 1]; t++) {
        const int sidx = hent[t] / 6;
        const double w = is_w[hent[t]];
        const double u = pxy[2 * p] - is_xy[2 * sidx], v = pxy[2 * p + 1] - is_xy[2 * sidx + 1];
        const double *z = zs + 6 * sidx;
        // grad m: (0,0) (1,0) (0,1) (2u,0) (v,u) (0,2v)
        gx -= w * (z[1] + 2.0 * u * z[3] + v * z[4]);
        gy -= w * (z[2] + u * z[4] + 2.0 * v * z[5]);
    }
    gpos[2 * p] += gx;
    gpos[2 * p + 1] += gy;
}

// Eq. 9 weights of ring node r: biquadratic Lagrange weights l_a(fx) l_b(fy)
// of its offset from the nearest lattice node (held: a moved node keeps its
// donors); add their position derivatives contracted with dJ/dw.
__global__ void k_adj_eq9_nodes(const int *perm, int ring_start, int n_ring, const double *pxy, const double *lw9,
                                double *gpos)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_ring) return;
    const int p = perm[ring_start + r];
    const double qx = pxy[2 * p], qy = pxy[2 * p + 1];
    const double fx = qx - floor(qx + 0.5), fy = qy - floor(qy + 0.5);
    const double lx[3] = {0.5 * fx * (fx - 1.0), 1.0 - fx * fx, 0.5 * fx * (fx + 1.0)};
    const double ly[3] = {0.5 * fy * (fy - 1.0), 1.0 - fy * fy, 0.5 * fy * (fy + 1.0)};
    const double dx[3] = {fx - 0.5, -2.0 * fx, fx + 0.5}, dy[3] = {fy - 0.5, -2.0 * fy, fy + 0.5};
    double gx = 0.0, gy = 0.0;
    for (int b = 0; b < 3; b++)
        for (int a = 0; a < 3; a++) {
            const double lw = lw9[9 * r + 3 * b + a];
            gx += lw * dx[a] * ly[b];
            gy += lw * lx[a] * dy[b];
        }
    gpos[2 * p] += gx;
    gpos[2 * p + 1] += gy;
}

// posed-frame gradient -> input frame (x_posed - p = R (x - p))
__global__ void k_adj_frame(const double *gpos, int n, double ca, double sa, double *grad_xy)
{
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    if (X >= n) return;
    const double gx = gpos[2 * X], gy = gpos[2 * X + 1];
    grad_xy[2 * size_t(X)] = ca * gx - sa * gy;
    grad_xy[2 * size_t(X) + 1] = sa * gx + ca * gy;
}

}  // namespace

void launch_adj_geometry(const AdjTables &A, int n, const double *gc, const double *gM, int Np, double wd, double wl,
                         double inv_q, double ca, double sa, double px, double py, double *scratch, double *grad_xy,
                         double *daoa, cudaStream_t s)
{
    double *abar = scratch, *h = scratch + n, *gpos = h + 2 * size_t(std::max(1, A.n_edges));
    k_adj_abar<<<(n + 127) / 128, 128, 0, s>>>(A.prow, A.pcoef, gc, A.parea, n, abar);
    if (A.n_edges > 0)
        k_adj_wall_normal<<<(A.n_edges + 127) / 128, 128, 0, s>>>(gM, Np, A.inv, A.iwea, A.iweb, A.n_edges, wd, wl,
                                                                 inv_q, 0, h);
    k_adj_shape<<<(n + 127) / 128, 128, 0, s>>>(A, n, gc, abar, h, ca, sa, gpos, grad_xy);
    k_adj_aoa<<<1, 256, 0, s>>>(A.pxy, gpos, n, ca, sa, px, py, daoa);
}

void launch_adj_value(const AdjTables &A, const double *g, int Np, double wd, double wl, double inv_q, double *J,
                      cudaStream_t s)
{
    k_adj_value<<<1, 256, 0, s>>>(g, Np, A.wea, A.web, A.wn, A.n_edges, wd, wl, inv_q, J);
}

void launch_adj_terminal(const AdjTables &A, const double *g, int Np, int n, double wd, double wl, double inv_q,
                         double *lam, cudaStream_t s, bool add)
{
    k_adj_terminal<<<(n + 127) / 128, 128, 0, s>>>(g, Np, n, A.wptr, A.wedge, A.wea, A.web, A.wn, wd, wl, inv_q,
                                                  add ? 1 : 0, lam);
}

void launch_fv_adjoint(const AdjTables &A, const double *g, int Np, int n, double csP, int n_wall, int ring_start,
                       int star, double dt, double dt_tau, const double *lam_in, double *lam_out, double *gcoef,
                       double *scratch, cudaStream_t s)
{
    double *mu = scratch, *sig = scratch + size_t(9) * Np, *E = scratch + size_t(18) * Np;
    const int blocks = (n + 127) / 128;
    k_adj_rows<<<blocks, 128, 0, s>>>(g, Np, n, A.rp, A.rcol, A.rcoef, csP, n_wall, ring_start, star, lam_in, mu, sig,
                                      E);
    k_adj_gather<<<blocks, 128, 0, s>>>(g, Np, n, A.rp, A.rcoef, A.rcsr, A.tp, A.trow, A.tpos, ring_start, star, dt,
                                        dt_tau, mu, sig, E, lam_out, gcoef);
}

void launch_adj_populations(const AdjTables &A, const double *g, int Np, int n, const double *lam, double *grad,
                            cudaStream_t s)
{
    k_adj_populations<<<(n + 127) / 128, 128, 0, s>>>(g, Np, n, A.perm, lam, grad);
}

}  // namespace hlbm

namespace hlbm {

void launch_adj_collide(const DevLevel &l, const double *f, int P, double *lam, cudaStream_t s)
{
    const dim3 grid((l.nx + 127) / 128, l.ny);
    const double omega = 1.0 / l.tau;
    if (P == 0) k_adj_collide<0><<<grid, 128, 0, s>>>(f, l.nx, l.ny, l.pitch, l.stride, omega, l.hx0, l.hx1, lam);
    else k_adj_collide<1><<<grid, 128, 0, s>>>(f, l.nx, l.ny, l.pitch, l.stride, omega, l.hx0, l.hx1, lam);
}

void launch_adj_outer_bc(const DevLevel &l, const double *f, int P, double u0, double *lam, cudaStream_t s)
{
    const dim3 grid((l.nx + 127) / 128, l.ny - 2);
    const int nper = 2 * l.nx + 2 * (l.ny - 2);
    if (P == 0) {
        k_adj_bc_gather<0><<<grid, 128, 0, s>>>(f, l.nx, l.ny, l.pitch, l.stride, u0, lam);
        k_adj_bc_clear<0><<<(nper + 127) / 128, 128, 0, s>>>(l.nx, l.ny, l.pitch, l.stride, lam);
    } else {
        k_adj_bc_gather<1><<<grid, 128, 0, s>>>(f, l.nx, l.ny, l.pitch, l.stride, u0, lam);
        k_adj_bc_clear<1><<<(nper + 127) / 128, 128, 0, s>>>(l.nx, l.ny, l.pitch, l.stride, lam);
    }
}

void launch_adj_ring_lattice(const DevLevel &l, const double *f, int P, const AdjTables &A, const double *ring_w,
                             const double *lamQ, int n_ring, double *lam, cudaStream_t s)
{
    const dim3 grid((l.nx + 127) / 128, l.ny);
    if (P == 0)
        k_adj_ring_lattice<0><<<grid, 128, 0, s>>>(f, l.nx, l.ny, l.pitch, l.stride, A.lptr, A.lent, ring_w, lamQ,
                                                  n_ring, lam);
    else
        k_adj_ring_lattice<1><<<grid, 128, 0, s>>>(f, l.nx, l.ny, l.pitch, l.stride, A.lptr, A.lent, ring_w, lamQ,
                                                  n_ring, lam);
}

void launch_adj_hole(const DevLevel &l, const DevMesh &m, const AdjTables &A, const double *g, int P, double *lam,
                     double *lamq, double *lam_g, cudaStream_t s, double *lw6)
{
    if (m.n_is == 0) return;
    const double scale4 = 2.0 * (l.tau - 1.0) / (2.0 * l.tau - 1.0);
    const int b = (m.n_is + 127) / 128;
    if (P == 0)
        k_adj_hole_q<0><<<b, 128, 0, s>>>(g, m.Np, m.is_n, m.is_don, (const double *)m.is_w, m.n_is, scale4, l.pitch,
                                          l.stride, lam, lamq, lw6);
    else
        k_adj_hole_q<1><<<b, 128, 0, s>>>(g, m.Np, m.is_n, m.is_don, (const double *)m.is_w, m.n_is, scale4, l.pitch,
                                          l.stride, lam, lamq, lw6);
    k_adj_hole_mesh<<<(m.n + 127) / 128, 128, 0, s>>>(g, m.Np, m.n, A.hptr, A.hent, (const double *)m.is_w, lamq,
                                                      m.n_is, lam_g);
}

void launch_adj_ring_rows(const DevMesh &m, double scale5, double wa, double wb, double *lam_g, double *lamQ0,
                          double *lamQ1, cudaStream_t s)
{
    if (m.n_ring == 0) return;
    k_adj_ring_rows<<<(m.n_ring + 127) / 128, 128, 0, s>>>(lam_g, m.Np, m.ring_start, m.n_ring, scale5, wa, wb,
                                                          lamQ0, lamQ1);
}

void launch_adj_lattice_out(const DevLevel &l, const double *lam, int P, double *grad, cudaStream_t s)
{
    const dim3 grid((l.nx + 127) / 128, l.ny);
    if (P == 0) k_adj_lattice_out<0><<<grid, 128, 0, s>>>(lam, l.nx, l.ny, l.pitch, l.stride, l.hx0, l.hx1, grad);
    else k_adj_lattice_out<1><<<grid, 128, 0, s>>>(lam, l.nx, l.ny, l.pitch, l.stride, l.hx0, l.hx1, grad);
}

}  // namespace hlbm

namespace hlbm {

void launch_adj_snapshot(const DevLevel &l, const double *f, int P, const double *lamS, double *lam, cudaStream_t s)
{
    const dim3 grid((l.cmx + 2 + 127) / 128, l.cmy + 2);
    if (P == 0) k_adj_snapshot<0><<<grid, 128, 0, s>>>(f, l.pitch, l.stride, l.cox, l.coy, l.cmx, l.cmy, lamS, l.band_n, lam);
    else k_adj_snapshot<1><<<grid, 128, 0, s>>>(f, l.pitch, l.stride, l.cox, l.coy, l.cmx, l.cmy, lamS, l.band_n, lam);
}

void launch_adj_prolong(const DevLevel &p, const DevLevel &l, int P, double theta, const double *A, const double *B,
                        const int *pp, const int *pk, const double *pw, double *lam, double *lamq, double *lamA,
                        double *lamB, cudaStream_t s)
{
    const int nper = 2 * l.nx + 2 * (l.ny - 2);
    const double scale = l.tau / (2.0 * p.tau);
    if (P == 0)
        k_adj_prolong_q<0><<<(nper + 127) / 128, 128, 0, s>>>(l.nx, l.ny, l.pitch, l.stride, A, B, p.band_n, p.cmx,
                                                              p.cmy, theta, scale, lam, lamq);
    else
        k_adj_prolong_q<1><<<(nper + 127) / 128, 128, 0, s>>>(l.nx, l.ny, l.pitch, l.stride, A, B, p.band_n, p.cmx,
                                                              p.cmy, theta, scale, lam, lamq);
    k_adj_prolong_band<<<(p.band_n + 127) / 128, 128, 0, s>>>(pp, pk, pw, lamq, nper, p.band_n, theta, lamA, lamB);
}

void launch_adj_restrict(const DevLevel &p, const DevLevel &l, int PC, int PF, const double *ff, double *lamc,
                         double *lamf, cudaStream_t s)
{
    if (p.cmx < 2 || p.cmy < 2) return;
    const dim3 grid((p.cmx - 1 + 127) / 128, p.cmy - 1);
    const double scale = 2.0 * p.tau / l.tau;
#define HLBM_ADJ_RESTRICT(A_, B_)                                                                                    \
    k_adj_restrict<A_, B_><<<grid, 128, 0, s>>>(ff, p.pitch, p.stride, l.pitch, l.stride, p.cox, p.coy, p.cmx, p.cmy, \
                                                scale, p.hx0, p.hx1, lamc, lamf)
    if (PC == 0 && PF == 0) HLBM_ADJ_RESTRICT(0, 0);
    else if (PC == 0) HLBM_ADJ_RESTRICT(0, 1);
    else if (PF == 0) HLBM_ADJ_RESTRICT(1, 0);
    else HLBM_ADJ_RESTRICT(1, 1);
#undef HLBM_ADJ_RESTRICT
}

}  // namespace hlbm

namespace hlbm {

void launch_adj_ring_weights(const DevLevel &l, const DevMesh &m, const double *f, int P, const double *lamQ,
                             double *lw9, cudaStream_t s)
{
    if (m.n_ring == 0) return;
    const int b = (m.n_ring + 127) / 128;
    if (P == 0) k_adj_ring_weights<0><<<b, 128, 0, s>>>(f, l.pitch, l.stride, m.ring_don, lamQ, m.n_ring, lw9);
    else k_adj_ring_weights<1><<<b, 128, 0, s>>>(f, l.pitch, l.stride, m.ring_don, lamQ, m.n_ring, lw9);
}

void launch_adj_geometry_coupled(const AdjTables &A, const DevMesh &m, int n, const double *gc, const double *hacc,
                                 const double *lw6, const double *lw9, double ca, double sa, double px, double py,
                                 double *scratch, double *grad_xy, double *daoa, cudaStream_t s)
{
    // scratch: abar [n], gpos [2 n], zs [6 n_is]
    double *abar = scratch, *gpos = scratch + n, *zs = gpos + 2 * size_t(n);
    const int b = (n + 127) / 128;
    k_adj_abar<<<b, 128, 0, s>>>(A.prow, A.pcoef, gc, A.parea, n, abar);
    k_adj_shape<<<b, 128, 0, s>>>(A, n, gc, abar, hacc, ca, sa, gpos, nullptr);
    if (m.n_is > 0) {
        k_adj_eq8_solve<<<(m.n_is + 127) / 128, 128, 0, s>>>(A.isd_in, A.is_xy, A.pxy, lw6, m.n_is, zs);
        k_adj_eq8_nodes<<<b, 128, 0, s>>>(A.hptr, A.hent, A.perm, (const double *)m.is_w, A.is_xy, A.pxy, zs, n,
                                          gpos);
    }
    if (m.n_ring > 0)
        k_adj_eq9_nodes<<<(m.n_ring + 127) / 128, 128, 0, s>>>(A.perm, m.ring_start, m.n_ring, A.pxy, lw9, gpos);
    if (grad_xy) k_adj_frame<<<b, 128, 0, s>>>(gpos, n, ca, sa, grad_xy);
    k_adj_aoa<<<1, 256, 0, s>>>(A.pxy, gpos, n, ca, sa, px, py, daoa);
}

}  // namespace hlbm

namespace hlbm {

void launch_adj_wall_normal(const AdjTables &A, const double *g, int Np, double wd, double wl, double inv_q,
                            double *hacc, cudaStream_t s)
{
    if (A.n_edges > 0)
        k_adj_wall_normal<<<(A.n_edges + 127) / 128, 128, 0, s>>>(g, Np, A.inv, A.iwea, A.iweb, A.n_edges, wd, wl,
                                                                 inv_q, 1, hacc);
}

}  // namespace hlbm
