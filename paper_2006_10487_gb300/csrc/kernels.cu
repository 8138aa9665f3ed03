// CUDA kernels of the HLBM step for sm_103a.
//
// Storage is deviations d_i = f_i - w_i (float or double); arithmetic is in
// the storage type.  Every kernel is a pure gather (each thread writes only
// its own outputs), so results are deterministic; no atomics are used (the
// bounds-checked build, HLBM_DEBUG, counts violations with atomics).
//
// Paper passages: Eq. 1-2 (lattice), Eq. 3 (finite volume), Eq. 4-9 (overlap
// coupling), Section 4 (refinement boxes, wall, outer conditions),
// Eq. 10-11 (forces).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "hlbm_device.h"

namespace hlbm {
namespace {

// ------------------------------------------------------ bounds checks -----
// Built with -DHLBM_DEBUG, every table-driven or computed index into a lattice
// level, the mesh state, a tile's staged shared memory or a band snapshot is
// checked against its extent: a violation is counted (site bit in d_bounds[1])
// and the access goes to index 0 instead, so the run stays in bounds and the
// host reads the count (hlbm_info "bounds_violations").  Release builds
// compile the checks away.
enum BoundsSite { kSiteLattice = 0, kSiteMesh = 1, kSiteStaged = 2, kSiteEntry = 3, kSiteBand = 4 };
#ifdef HLBM_DEBUG
__device__ unsigned int d_bounds[2];  // violations, bit mask of sites
template <typename I> __device__ __forceinline__ I checked(I i, I n, int site)
{
    bool ok = i < n;
    if constexpr (std::is_signed_v<I>) ok = ok && i >= I(0);
    if (ok) return i;
    atomicAdd(&d_bounds[0], 1u);
    atomicOr(&d_bounds[1], 1u << site);
    return I(0);
}
#define HLBM_CHK(i, n, site) checked<std::decay_t<decltype(i)>>((i), std::decay_t<decltype(i)>(n), (site))
#else
#define HLBM_CHK(i, n, site) (i)
#endif

// ---------------------------------------------------------------- D2Q9 -----
// order: (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
__host__ __device__ __forceinline__ constexpr int cx(int i)
{
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int cy(int i)
{
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int opp(int i)
{
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
template <typename T> __device__ __forceinline__ T wq(int i)
{
    return i == 0 ? T(4.0 / 9.0) : (i <= 4 ? T(1.0 / 9.0) : T(1.0 / 36.0));
}

// Eq. 2 in deviation form: f^eq_i - w_i = w_i [(rho - 1) + rho (3 cu + 9/2 cu^2 - 3/2 u.u)].
template <typename T> __device__ __forceinline__ T deq(int i, T rho, T ux, T uy)
{
    T cu = T(cx(i)) * ux + T(cy(i)) * uy;
    T uu = ux * ux + uy * uy;
    return wq<T>(i) * ((rho - T(1)) + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu));
}

template <typename T> __device__ __forceinline__ void moments(const T d[9], T &rho, T &ux, T &uy)
{
    T s = 0, mx = 0, my = 0;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        s += d[i];
        mx += T(cx(i)) * d[i];
        my += T(cy(i)) * d[i];
    }
    rho = T(1) + s;
    ux = mx / rho;
    uy = my / rho;
}

// q = (rho, ux, uy, f^neq_0..8)
template <typename T> __device__ __forceinline__ void to_q(const T d[9], T q[12])
{
    moments(d, q[0], q[1], q[2]);
#pragma unroll
    for (int i = 0; i < 9; i++) q[3 + i] = d[i] - deq<T>(i, q[0], q[1], q[2]);
}

// d = f^eq(rho, u) - w + scale * f^neq
template <typename T> __device__ __forceinline__ void from_q(const T q[12], T scale, T d[9])
{
#pragma unroll
    for (int i = 0; i < 9; i++) d[i] = deq<T>(i, q[0], q[1], q[2]) + scale * q[3 + i];
}

// Mesh state, plane-major g[9][Np]: plane 0 = rho - 1, planes 1-2 = u,
// planes 3-8 = f^neq_3..8.  f^neq_0..2 follow from the zero mass and momentum
// of the non-equilibrium part:
//   f^neq_1 = f^neq_3 - f^neq_5 + f^neq_6 + f^neq_7 - f^neq_8
//   f^neq_2 = f^neq_4 - f^neq_5 - f^neq_6 + f^neq_7 + f^neq_8
//   f^neq_0 = -(f^neq_1 + ... + f^neq_8)
template <typename T> __device__ __forceinline__ void neq_complete(T nq[9])
{
    nq[1] = nq[3] - nq[5] + nq[6] + nq[7] - nq[8];
    nq[2] = nq[4] - nq[5] - nq[6] + nq[7] + nq[8];
    nq[0] = -(nq[1] + nq[2] + nq[3] + nq[4] + nq[5] + nq[6] + nq[7] + nq[8]);
}

template <typename T>
__device__ __forceinline__ void load_mesh(const T *__restrict__ g, int Np, int k, T &r1, T &ux, T &uy, T nq[9])
{
    k = HLBM_CHK(k, Np, kSiteMesh);
    r1 = g[k];
    ux = g[size_t(Np) + k];
    uy = g[size_t(2) * Np + k];
#pragma unroll
    for (int i = 3; i < 9; i++) nq[i] = g[size_t(i) * Np + k];
    neq_complete(nq);
}

// q = (rho, ux, uy, f^neq_0..8) of a mesh node
template <typename T> __device__ __forceinline__ void mesh_q(const T *__restrict__ g, int Np, int k, T q[12])
{
    T r1;
    load_mesh(g, Np, k, r1, q[1], q[2], q + 3);
    q[0] = T(1) + r1;
}

// E_i(u) = 1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u  (f^eq_i = w_i rho E_i(u))
template <typename T> __device__ __forceinline__ T Efun(int i, T ux, T uy)
{
    T cu = T(cx(i)) * ux + T(cy(i)) * uy;
    return T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * (ux * ux + uy * uy);
}

// f^eq_i(rho_b + drho, u_b + du) - f^eq_i(rho_b, u_b) through moment differences:
//   w_i [drho E_i(u_b) + rho_a (3 c.du + 9/2 (c.du)(c.(u_a + u_b)) - 3/2 du.(u_a + u_b))]
template <typename T>
__device__ __forceinline__ T feq_diff(int i, T Eb, T drho, T rho_a, T dux, T duy, T sux, T suy)
{
    T cdu = T(cx(i)) * dux + T(cy(i)) * duy, csu = T(cx(i)) * sux + T(cy(i)) * suy;
    return wq<T>(i) * (drho * Eb + rho_a * (T(3) * cdu + T(4.5) * cdu * csu - T(1.5) * (dux * sux + duy * suy)));
}

// AA-pattern addressing.  State of node n at parity p:
//   p = 0: plane i at n;  p = 1: plane opp(i) at n - c_i.
// A collision at parity p writes its post-collision value c_i-bound to
//   p = 0: plane opp(i) at n;  p = 1: plane i at n + c_i.
template <int P> __device__ __forceinline__ size_t st_idx(int i, size_t n, int pitch, size_t stride)
{
    if (P == 0) return size_t(i) * stride + HLBM_CHK(n, stride, kSiteLattice);
    return size_t(opp(i)) * stride + HLBM_CHK(n - cx(i) - ptrdiff_t(cy(i)) * pitch, stride, kSiteLattice);
}
template <int P> __device__ __forceinline__ size_t wr_idx(int i, size_t n, int pitch, size_t stride)
{
    if (P == 0) return size_t(opp(i)) * stride + HLBM_CHK(n, stride, kSiteLattice);
    return size_t(i) * stride + HLBM_CHK(n + cx(i) + ptrdiff_t(cy(i)) * pitch, stride, kSiteLattice);
}

__device__ __forceinline__ size_t node(int x, int y, int pitch) { return size_t(y + 1) * pitch + x + 1; }

// Lattice storage.  float / double levels store d_i = f_i - w_i as is.  FP16S
// levels store the 16-bit float (d_i - s_i) / w_i with s_i = f^eq_i(1, (u0, 0))
// - w_i, the free stream: small relative deviations, so that the 11-bit
// significand is spent where the flow differs from the free stream.
template <typename T> __device__ __forceinline__ T inv_w(int i)
{
    return i == 0 ? T(9.0 / 4.0) : (i <= 4 ? T(9.0) : T(36.0));
}
template <typename S> struct Codec {
    template <typename T> __device__ static T get(const S *f, size_t k, int, const LatShift &) { return T(f[k]); }
    template <typename T> __device__ static void put(S *f, size_t k, int, T v, const LatShift &) { f[k] = S(v); }
};
template <> struct Codec<__half> {
    template <typename T> __device__ static T get(const __half *f, size_t k, int i, const LatShift &sh)
    {
        return wq<T>(i) * T(__half2float(f[k])) + T(sh.s[i]);
    }
    template <typename T> __device__ static void put(__half *f, size_t k, int i, T v, const LatShift &sh)
    {
        f[k] = __float2half_rn(float((v - T(sh.s[i])) * inv_w<T>(i)));
    }
};

template <typename T, typename S, int P>
__device__ __forceinline__ void load_state(const S *f, size_t n, int pitch, size_t stride, T d[9], const LatShift &sh)
{
#pragma unroll
    for (int i = 0; i < 9; i++) d[i] = Codec<S>::template get<T>(f, st_idx<P>(i, n, pitch, stride), i, sh);
}
template <typename T, typename S, int P>
__device__ __forceinline__ void store_state(S *f, size_t n, int pitch, size_t stride, const T d[9], const LatShift &sh)
{
#pragma unroll
    for (int i = 0; i < 9; i++) Codec<S>::template put<T>(f, st_idx<P>(i, n, pitch, stride), i, d[i], sh);
}

// splitmix64 (Steele, Lea and Flood): uniform deviate in [-1, 1)
__device__ __forceinline__ double deviate(uint64_t seed, uint64_t grid, uint64_t idx)
{
    uint64_t z = (seed ^ (grid << 40) ^ idx) + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return double(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

// -------------------------------------------------------------- kernels ----
// Initial lattice state: f = f^eq(1 + perturb xi, (u0, 0)); hole nodes and the
// halo hold NaN so that any read of them shows up in the results.
template <typename T, typename S>
__global__ void k_init_level(S *f, int nx, int ny, int pitch, size_t stride, const int *hx0, const int *hx1,
                             uint64_t seed, int grid, double perturb, double u0, LatShift sh)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x - 1, y = int(blockIdx.y) - 1;
    if (x > nx) return;
    size_t n = size_t(y + 1) * pitch + x + 1;
    bool inside = x >= 0 && y >= 0 && x < nx && y < ny;
    bool hole = inside && hx0 && x >= hx0[y] && x < hx1[y];
    if (!inside || hole) {
#pragma unroll
        for (int i = 0; i < 9; i++) Codec<S>::template put<T>(f, size_t(i) * stride + n, i, T(NAN), sh);
        return;
    }
    double rho = 1.0 + perturb * deviate(seed, uint64_t(grid), uint64_t(y) * nx + x);
#pragma unroll
    for (int i = 0; i < 9; i++) Codec<S>::template put<T>(f, size_t(i) * stride + n, i, T(deq<double>(i, rho, u0, 0.0)), sh);
}

// Eq. 1: BGK collision and (implicit, AA-pattern) streaming on one level.
// Each thread treats kCollideNodes nodes of one row, kCollideThreads apart
// (coalesced per node), loading all their populations before any store so
// that the loads of every node are in flight together (the in-place layout
// keeps the compiler from moving one node's loads above another's stores).
constexpr int kCollideThreads = 128, kCollideNodes = 4;
template <typename T, typename S, int P>
__global__ void __launch_bounds__(kCollideThreads) k_collide(S *__restrict__ f, int nx, int ny, int pitch,
                                                             size_t stride, T omega, const int *__restrict__ hx0,
                                                             const int *__restrict__ hx1, LatShift sh)
{
    const int y = blockIdx.y;
    const int x0 = blockIdx.x * (kCollideThreads * kCollideNodes) + threadIdx.x;
    const int h0 = hx0 ? hx0[y] : 0, h1 = hx0 ? hx1[y] : 0;
    bool live[kCollideNodes];
    T d[kCollideNodes][9];
#pragma unroll
    for (int j = 0; j < kCollideNodes; j++) {
        const int x = x0 + j * kCollideThreads;
        live[j] = x < nx && !(x >= h0 && x < h1);
        if (live[j]) load_state<T, S, P>(f, node(x, y, pitch), pitch, stride, d[j], sh);
    }
#pragma unroll
    for (int j = 0; j < kCollideNodes; j++) {
        if (!live[j]) continue;
        const size_t n = node(x0 + j * kCollideThreads, y, pitch);
        T rho, ux, uy;
        moments(d[j], rho, ux, uy);
#pragma unroll
        for (int i = 0; i < 9; i++) {
            T post = d[j][i] - omega * (d[j][i] - deq<T>(i, rho, ux, uy));
            Codec<S>::template put<T>(f, wr_idx<P>(i, n, pitch, stride), i, post, sh);
        }
    }
}

// Outer conditions on the level-0 perimeter (Section 4), written as the
// state at parity P: every perimeter node copies the state of its nearest
// interior node n (coordinates clamped to the interior) with
//   inlet (x = 0):        f^eq(rho_n, (u0, 0)) + f^neq_n
//   outlet (x = nx - 1):  f^eq(1, u_n) + f^neq_n
//   top / bottom:         f_n
template <typename T, typename S, int P>
__global__ void k_outer_bc(S *f, int nx, int ny, int pitch, size_t stride, T u0, LatShift sh)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int nper = 2 * nx + 2 * (ny - 2);
    if (k >= nper) return;
    int x, y;
    if (k < nx) { x = k; y = 0; }
    else if (k < 2 * nx) { x = k - nx; y = ny - 1; }
    else if (k < 2 * nx + ny - 2) { x = 0; y = k - 2 * nx + 1; }
    else { x = nx - 1; y = k - 2 * nx - (ny - 2) + 1; }
    int xn = min(max(x, 1), nx - 2), yn = min(max(y, 1), ny - 2);
    T d[9];
    load_state<T, S, P>(f, node(xn, yn, pitch), pitch, stride, d, sh);
    if (x == 0 || x == nx - 1) {
        T q[12];
        to_q(d, q);
        if (x == 0) { q[1] = u0; q[2] = T(0); }
        else q[0] = T(1);
        from_q(q, T(1), d);
    }
    store_state<T, S, P>(f, node(x, y, pitch), pitch, stride, d, sh);
}

// Coarse node of band entry b: the lines y = coy and y = coy + cmy for
// x in [cox - 1, cox + cmx], then x = cox and x = cox + cmx for
// y in [coy - 1, coy + cmy].
__device__ __forceinline__ void band_node(int b, int cox, int coy, int cmx, int cmy, int &X, int &Y)
{
    int w = cmx + 2, h = cmy + 2;
    if (b < w) { X = cox - 1 + b; Y = coy; }
    else if (b < 2 * w) { X = cox - 1 + b - w; Y = coy + cmy; }
    else if (b < 2 * w + h) { X = cox; Y = coy - 1 + b - 2 * w; }
    else { X = cox + cmx; Y = coy - 1 + b - 2 * w - h; }
}

// (rho, u, f^neq) of the parent level along its child's boundary band.
template <typename T, typename S, int P>
__global__ void k_snapshot(const S *f, int pitch, size_t stride, int cox, int coy, int cmx, int cmy, T *snap,
                           int band_n, LatShift sh)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= band_n) return;
    int X, Y;
    band_node(b, cox, coy, cmx, cmy, X, Y);
    T d[9], q[12];
    load_state<T, S, P>(f, node(X, Y, pitch), pitch, stride, d, sh);
    to_q(d, q);
#pragma unroll
    for (int m = 0; m < 12; m++) snap[size_t(m) * band_n + b] = q[m];
}

// Refinement coarse -> fine (Section 4): the fine boundary ring at parity P
// takes f^eq(rho, u) + tau_f / (2 tau_c) f^neq from the parent band, linear
// in time (theta) and, midway between coarse nodes, quadratic along the
// ring through coarse nodes X-1, X, X+1 (weights -1/8, 3/4, 3/8).
template <typename T, typename S, int P>
__global__ void k_prolong(S *f, int nx, int ny, int pitch, size_t stride, const T *snapA, const T *snapB,
                          int band_n, int cox, int coy, int cmx, int cmy, T theta, T scale, LatShift sh)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int nper = 2 * nx + 2 * (ny - 2);
    if (k >= nper) return;
    int i, j;
    if (k < nx) { i = k; j = 0; }
    else if (k < 2 * nx) { i = k - nx; j = ny - 1; }
    else if (k < 2 * nx + ny - 2) { i = 0; j = k - 2 * nx + 1; }
    else { i = nx - 1; j = k - 2 * nx - (ny - 2) + 1; }
    int w = cmx + 2, h = cmy + 2;
    int base, pos, odd;
    if (j == 0 || j == ny - 1) {  // bottom / top line, along x
        base = (j == 0) ? 0 : w;
        pos = (i >> 1) + 1;  // band position of coarse x = cox + floor(i/2)
        odd = i & 1;
    } else {  // left / right line, along y
        base = 2 * w + ((i == 0) ? 0 : h);
        pos = (j >> 1) + 1;
        odd = j & 1;
    }
    T q[12];
#pragma unroll
    for (int m = 0; m < 12; m++) q[m] = T(0);
    const int nd = odd ? 3 : 1;
    for (int t = 0; t < nd; t++) {
        int b = HLBM_CHK(base + pos + (odd ? t - 1 : 0), band_n, kSiteBand);
        T wk = odd ? (t == 0 ? T(-0.125) : (t == 1 ? T(0.75) : T(0.375))) : T(1);
#pragma unroll
        for (int m = 0; m < 12; m++)
            q[m] += wk * ((T(1) - theta) * snapA[size_t(m) * band_n + b] + theta * snapB[size_t(m) * band_n + b]);
    }
    T d[9];
    from_q(q, scale, d);
    store_state<T, S, P>(f, node(i, j, pitch), pitch, stride, d, sh);
}

// Refinement fine -> coarse: coarse nodes at least one cell inside the child
// box take the coincident fine state with f^neq scaled by 2 tau_c / tau_f.
template <typename T, typename S, int PC, int PF>
__global__ void k_restrict(S *fc, int pitch_c, size_t stride_c, const S *ff, int pitch_f, size_t stride_f, int cox,
                           int coy, int cmx, int cmy, T scale, const int *hx0, const int *hx1, LatShift sh)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (a >= cmx - 1) return;
    int X = cox + 1 + a, Y = coy + 1 + b;
    if (hx0 && X >= hx0[Y] && X < hx1[Y]) return;  // over the hole: not computed
    T d[9], q[12];
    load_state<T, S, PF>(ff, node(2 * (X - cox), 2 * (Y - coy), pitch_f), pitch_f, stride_f, d, sh);
    to_q(d, q);
    from_q(q, scale, d);
    store_state<T, S, PC>(fc, node(X, Y, pitch_c), pitch_c, stride_c, d, sh);
}

// Eq. 9: (rho, u, f^neq) at the unstructured interpolation nodes from their
// 3x3 lattice donors.  With star != 0 (after the lattice step) the kernel also
// sets the ring nodes of the read buffer to the Eq. 5-6 state at theta = 0:
// (rho, u, (1 - 1/(2 tau_s)) f^neq) of the data at t (Q0).
// 16 lanes per ring node: lane k < 9 takes donor k; xor-shuffle sum.
template <typename T, typename S, int P>
__global__ void k_ring_interp(const S *f, int pitch, size_t stride, const int *don, const T *w, int n_ring,
                              T *Q, const T *Q0, T *g, int Np, int ring_start, T scale5, int star, LatShift sh)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int r = t >> 4, k = t & 15;
    bool live = r < n_ring;
    int rr = live ? r : n_ring - 1;
    T acc[12];
#pragma unroll
    for (int m = 0; m < 12; m++) acc[m] = T(0);
    if (k < 9) {
        T d[9], q[12];
        load_state<T, S, P>(f, size_t(don[9 * rr + k]), pitch, stride, d, sh);
        to_q(d, q);
        T wk = w[9 * rr + k];
#pragma unroll
        for (int m = 0; m < 12; m++) acc[m] = wk * q[m];
    }
#pragma unroll
    for (int m = 0; m < 12; m++)
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
    if (!live) return;
#pragma unroll
    for (int m = 0; m < 12; m++)
        if (m == k) Q[size_t(m) * n_ring + r] = acc[m];
    if (star && k < 9) {
        // mesh state (rho - 1, u, (1 - 1/(2 tau_s)) f^neq) of the data at t
        // mesh plane k: rho - 1, ux, uy (q[0..2]) or f^neq_k (q[3 + k])
        T v = Q0[size_t(k < 3 ? k : 3 + k) * n_ring + r];
        g[size_t(k) * Np + HLBM_CHK(ring_start + r, Np, kSiteMesh)] = k == 0 ? v - T(1) : (k < 3 ? v : scale5 * v);
    }
}

// Eq. 4 with Eq. 8: post-collision state of the structured interpolation
// nodes from six unstructured donors, written where the collision at parity
// P would write it.  8 lanes per node: lane k < 6 takes donor k.
template <typename T, typename S, int P>
__global__ void k_hole_interp(S *f, int pitch, size_t stride, const int *is_n, const int *don, const T *w, int n_is,
                              const T *g, int Np, T scale4, LatShift sh)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int s = t >> 3, k = t & 7;
    bool live = s < n_is;
    int ss = live ? s : n_is - 1;
    T acc[12];
#pragma unroll
    for (int m = 0; m < 12; m++) acc[m] = T(0);
    if (k < 6) {
        int p = don[6 * ss + k];
        T q[12];
        mesh_q(g, Np, p, q);
        T wk = w[6 * ss + k];
#pragma unroll
        for (int m = 0; m < 12; m++) acc[m] = wk * q[m];
    }
#pragma unroll
    for (int m = 0; m < 12; m++)
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
    if (!live) return;
    size_t n = size_t(is_n[s]);
    // lane k writes population k (lane 0 also population 8)
#pragma unroll
    for (int i = 0; i < 9; i++)
        if ((i & 7) == k)
            Codec<S>::template put<T>(f, wr_idx<P>(i, n, pitch, stride), i,
                                      deq<T>(i, acc[0], acc[1], acc[2]) + scale4 * acc[3 + i], sh);
}

template <typename T> struct Ent;
template <> struct Ent<float> { using type = float4; };
template <> struct Ent<double> { using type = double4_32a; };

__device__ __forceinline__ void unpack(const float4 &e, float &sx, float &sy, float &c, int &col)
{
    sx = e.x; sy = e.y; c = e.z; col = __float_as_int(e.w);
}
__device__ __forceinline__ void unpack(const double4_32a &e, double &sx, double &sy, double &c, int &col)
{
    sx = e.x; sy = e.y; c = e.z; col = int(e.w);
}

// Packed pairs of FP32 values (two halves of one 64-bit register) for the
// paired FP32 arithmetic (f32x2) of sm_100 and later: element-wise, round to
// nearest; one instruction does two of the FV kernel's accumulations.
__device__ __forceinline__ unsigned long long pk2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Two FP32 values in one register pair, with the paired operations above.
struct F2 {
    unsigned long long v;
};
__device__ __forceinline__ F2 f2(float lo, float hi) { return {pk2(lo, hi)}; }
__device__ __forceinline__ F2 f2(float a) { return {pk2(a, a)}; }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return {add2(a.v, b.v)}; }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return {sub2(a.v, b.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return {mul2(a.v, b.v)}; }
__device__ __forceinline__ F2 fmaf2(F2 a, F2 b, F2 c) { return {fma2(a.v, b.v, c.v)}; }

// Eq. 3, one explicit sub-step on every mesh node (node-major gather over the
// sliced-ELL operator rows, no atomics), on the (rho, u, f^neq) state:
//   acc_i = dt sum_k (c_i . s_Pk) (g_i(P_k) - g_i(P)) - dt/tau_u sum_k C_Pk f^neq_i(P_k)
// with g(P_k) - g(P) = [f^eq(P_k) - f^eq(P)] + [f^neq(P_k) - f^neq(P)]
// (sum_k s_Pk = 0); then rho' = rho + sum acc, u' from the momentum and
// f^neq' = f^neq + acc - [f^eq(rho', u') - f^eq(rho, u)].  Wall rows take
// u' = 0 (no-slip: rho and f^neq kept); ring rows, unless this is the last
// sub-step, take the Eq. 5-6 state of the next sub-step (theta_next).
//
// The own node P carries no streaming term and collision weight C_PP = 11/18
// (the control-volume mean of its hat function, the same on every node), so
// the operator rows hold only the edge neighbours.
// Evaluation.  With (a_k, b_k) = dt s_Pk, the equilibrium part of the
// streaming sum, sum_k (c_i.(a_k, b_k)) [f^eq_i(P_k) - f^eq_i(P)], is a
// polynomial in the components of c_i:
//   w_i [ E_i(u_P) (c_x D_x + c_y D_y) + 3 (c_x^2 Q_xx + c_x c_y Q_xy + c_y^2 Q_yy)
//         + 9/2 (c_x M_x + c_y M_y + c_x^2 c_y M_xxy + c_x c_y^2 M_xyy)
//         - 3/2 (c_x L_x + c_y L_y) ]
// (c_x^3 = c_x for D2Q9), whose 13 moment sums over the neighbours (D, Q, M,
// L below, with drho, du = u_k - u_P, su = u_k + u_P) are accumulated once per
// neighbour; only the f^neq part is summed per population.
// Each block is one tile of kTileRows consecutive rows (a compact patch: rows
// are in Morton order).  Before the dependency wait (constant data only): one
// thread starts a bulk asynchronous copy (TMA) of the tile's operator entries
// (its consecutive slices, one contiguous block) into shared memory, and every
// thread loads the index of the staged node it gathers.  After the wait the
// states of every node the tile touches are staged in shared memory,
// plane-major: the tile's own rows (the first kTileRows places of its staged
// list) by nine bulk copies, one per plane, the other nodes (sorted, after
// them) by the threads' loads; then each thread treats one row, reading its
// entries and its neighbours from shared memory.  Within each 32-row slice the
// set-up orders the rows' entries so that one slot's reads spread over the
// shared-memory banks.
constexpr int kFvGroup = 2;
constexpr int kFvHaloRegs = 1;  // staged nodes beyond the tile's own rows gathered per thread from registers
constexpr int kFvPrefetchRegs = 1;  // nodes beyond a later tile's own rows prefetched into L2, per thread
constexpr unsigned long long kWaitLimitNs = 500ull * 1000 * 1000;  // bounded waits give up after 0.5 s
constexpr int kFlagTimeout = 2;  // health flag bit: a device-side wait gave up

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for phase `parity` of the shared-memory mbarrier at `bar`, for at most
// kWaitLimitNs; returns false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const unsigned long long t0 = globaltimer();
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
        if (globaltimer() - t0 > kWaitLimitNs) return false;
    }
}

// One row of the FP64 sub-step: the sums over the row's neighbours (13 moment
// sums of the f^eq differences, 16 sums of the stored f^neq planes) and the
// closed-form update (see k_fv); the staged list holds nine planes.
template <typename T>
__device__ __forceinline__ void fv_row_f64(const T *__restrict__ sh, int hn, int own_pos,
                                           const typename Ent<T>::type *__restrict__ se, int base, int len, T dt_tau,
                                           int n_ent, T &r1, T &ux, T &uy, T nq[9])
{
    (void)n_ent;
    // own state from the staged list
    T r1P, uPx, uPy, nP[9];
    {
        const int p = HLBM_CHK(own_pos, hn, kSiteStaged);
        r1P = sh[p];
        uPx = sh[hn + p];
        uPy = sh[2 * hn + p];
#pragma unroll
        for (int i = 3; i < 9; i++) nP[i] = sh[i * hn + p];
        neq_complete(nP);
    }
    // own node: no streaming term (g(P) - g(P) = 0), collision weight C_PP = 11/18
    // f^neq part of the sums, over the six stored planes j = 3..8 only:
    //   U_j = sum_k a_k n_j(P_k), V_j = sum_k b_k n_j(P_k), W_j = sum_k cs_k n_j(P_k)
    // (U_4 and V_3 are never needed: c_4x = c_3y = 0); planes 0-2 follow at the
    // end from the same linear constraints that complete f^neq.
    T U3 = 0, U5 = 0, U6 = 0, U7 = 0, U8 = 0, V4 = 0, V5 = 0, V6 = 0, V7 = 0, V8 = 0;
    T W3 = 0, W4 = 0, W5 = 0, W6 = 0, W7 = 0, W8 = 0;
    T Sa = 0, Sb = 0, Dx = 0, Dy = 0, Qxx = 0, Qyy = 0, Qxy = 0, Lx = 0, Ly = 0, Mx = 0, My = 0, Mxxy = 0, Mxyy = 0;
    for (int e0 = 0; e0 < len; e0 += kFvGroup) {
        T sx[kFvGroup], sy[kFvGroup], c[kFvGroup];
        int k[kFvGroup];
#pragma unroll
        for (int j = 0; j < kFvGroup; j++) {
            if (e0 + j < len) {
                unpack(se[HLBM_CHK(base + 32 * (e0 + j), n_ent, kSiteEntry)], sx[j], sy[j], c[j], k[j]);
                k[j] = HLBM_CHK(k[j], hn, kSiteStaged);
            } else {
                sx[j] = sy[j] = c[j] = T(0);
                k[j] = 0;
            }
        }
        T st[kFvGroup][9];
#pragma unroll
        for (int j = 0; j < kFvGroup; j++)
#pragma unroll
            for (int i = 0; i < 9; i++) st[j][i] = sh[i * hn + k[j]];
#pragma unroll
        for (int j = 0; j < kFvGroup; j++) {
            const T a = sx[j], b = sy[j], cs = c[j];  // dt s_Pk and (dt / tau_u) C_Pk
            const T drho = st[j][0] - r1P, rhok = T(1) + st[j][0];
            const T dux = st[j][1] - uPx, duy = st[j][2] - uPy, sux = st[j][1] + uPx, suy = st[j][2] + uPy;
            const T dus = dux * sux + duy * suy, ra = rhok * a, rb = rhok * b;
            const T xs = dux * suy + duy * sux;
            Sa += a;
            Sb += b;
            Dx += a * drho;
            Dy += b * drho;
            Qxx += ra * dux;
            Qyy += rb * duy;
            Qxy += ra * duy + rb * dux;
            Lx += ra * dus;
            Ly += rb * dus;
            Mx += ra * dux * sux;
            My += rb * duy * suy;
            Mxxy += ra * xs + rb * dux * sux;
            Mxyy += rb * xs + ra * duy * suy;
            const T *nk = st[j];
            U3 += a * nk[3]; U5 += a * nk[5]; U6 += a * nk[6]; U7 += a * nk[7]; U8 += a * nk[8];
            V4 += b * nk[4]; V5 += b * nk[5]; V6 += b * nk[6]; V7 += b * nk[7]; V8 += b * nk[8];
            W3 += cs * nk[3]; W4 += cs * nk[4]; W5 += cs * nk[5];
            W6 += cs * nk[6]; W7 += cs * nk[7]; W8 += cs * nk[8];
        }
    }
    // Update.  With acc_i = sum_k (c_i.(a_k, b_k) - cs_k) f^neq_i(P_k) + w_i eq_i
    // - f^neq_i(P) (c_i.(Sa, Sb) + dt/tau_u C_PP) the increment of population i,
    // its zeroth and first moments need no per-population sum: f^neq carries
    // no mass or momentum and the D2Q9 weights are isotropic to fourth order,
    //   drho = u_P.D + Q_xx + Q_yy
    //   djx  = D_x/3 + u_Px (u_P.D) + 3/2 M_x + 1/2 M_xyy - 1/2 L_x
    //          + sum_k (a_k Pi^neq_xx(P_k) + b_k Pi^neq_xy(P_k)) - (Sa Pi^neq_xx(P) + Sb Pi^neq_xy(P))
    // (djy likewise), with sum_k a_k Pi^neq_xx(P_k) = 2 (U3 + U6 + U7) and so
    // on.  The new f^neq is then needed for the stored planes 3..8 only;
    // opposite diagonals (5, 7) and (6, 8) share the even and odd parts of
    // eq_i and of the f^eq difference.
    const T csP = dt_tau * T(11.0 / 18.0);
    const T Pxx = nP[1] + nP[3] + nP[5] + nP[6] + nP[7] + nP[8];
    const T Pyy = nP[2] + nP[4] + nP[5] + nP[6] + nP[7] + nP[8];
    const T Pxy = nP[5] - nP[6] + nP[7] - nP[8];
    const T uD = uPx * Dx + uPy * Dy;
    const T drho = uD + Qxx + Qyy;
    const T djx = Dx * T(1.0 / 3.0) + uPx * uD + T(1.5) * Mx + T(0.5) * Mxyy - T(0.5) * Lx + T(2) * (U3 + U6 + U7) +
                  (V5 - V6 + V7 - V8) - (Sa * Pxx + Sb * Pxy);
    const T djy = Dy * T(1.0 / 3.0) + uPy * uD + T(1.5) * My + T(0.5) * Mxxy - T(0.5) * Ly + (U5 - U6 + U7 - U8) +
                  T(2) * (V4 + V7 + V8) - (Sb * Pyy + Sa * Pxy);
    r1 = r1P + drho;
    const T rho = T(1) + r1, irho = T(1) / rho;
    const T dux = (djx - drho * uPx) * irho, duy = (djy - drho * uPy) * irho;
    ux = uPx + dux;
    uy = uPy + duy;
    const T sx = ux + uPx, sy = uy + uPy;           // u' + u_P
    const T E0 = T(1) - T(1.5) * (uPx * uPx + uPy * uPy);
    const T ddot = T(1.5) * (dux * sx + duy * sy);  // 3/2 du.(u' + u_P)
    // [f^eq_c(rho', u') - f^eq_c(rho_P, u_P)] / w_c for a direction c with E = E_c(u_P)
    auto fd = [&](T E, T cdu, T csu) { return drho * E + rho * (T(3) * cdu + T(4.5) * cdu * csu - ddot); };
    {  // axis directions 3 (-1, 0) and 4 (0, -1)
        const T E3 = E0 - T(3) * uPx + T(4.5) * uPx * uPx;
        const T eq3 = -E3 * Dx + T(3) * Qxx - T(4.5) * Mx + T(1.5) * Lx;
        nq[3] = nP[3] - U3 - W3 + T(1.0 / 9.0) * eq3 + nP[3] * (Sa - csP) - T(1.0 / 9.0) * fd(E3, -dux, -sx);
        const T E4 = E0 - T(3) * uPy + T(4.5) * uPy * uPy;
        const T eq4 = -E4 * Dy + T(3) * Qyy - T(4.5) * My + T(1.5) * Ly;
        nq[4] = nP[4] - V4 - W4 + T(1.0 / 9.0) * eq4 + nP[4] * (Sb - csP) - T(1.0 / 9.0) * fd(E4, -duy, -sy);
    }
    {  // diagonals 5 (1, 1) and 7 (-1, -1)
        const T q = uPx + uPy, A = E0 + T(4.5) * q * q, B = T(3) * q;
        const T Pd = Dx + Dy, C = T(3) * (Qxx + Qxy + Qyy);
        const T Z = T(4.5) * (Mx + My + Mxxy + Mxyy) - T(1.5) * (Lx + Ly);
        const T odd = A * Pd + Z, even = B * Pd + C;  // eq5 = even + odd, eq7 = even - odd
        const T cdu = dux + duy, csu = sx + sy;
        nq[5] = nP[5] + U5 + V5 - W5 + T(1.0 / 36.0) * (even + odd) - nP[5] * (Sa + Sb + csP) -
                T(1.0 / 36.0) * fd(A + B, cdu, csu);
        nq[7] = nP[7] - U7 - V7 - W7 + T(1.0 / 36.0) * (even - odd) + nP[7] * (Sa + Sb - csP) -
                T(1.0 / 36.0) * fd(A - B, -cdu, -csu);
    }
    {  // diagonals 6 (-1, 1) and 8 (1, -1)
        const T q = uPy - uPx, A = E0 + T(4.5) * q * q, B = T(3) * q;
        const T Pd = Dy - Dx, C = T(3) * (Qxx - Qxy + Qyy);
        const T Z = T(4.5) * (-Mx + My + Mxxy - Mxyy) - T(1.5) * (Ly - Lx);
        const T odd = A * Pd + Z, even = B * Pd + C;  // eq6 = even + odd, eq8 = even - odd
        const T cdu = duy - dux, csu = sy - sx;
        nq[6] = nP[6] - U6 + V6 - W6 + T(1.0 / 36.0) * (even + odd) - nP[6] * (Sb - Sa + csP) -
                T(1.0 / 36.0) * fd(A + B, cdu, csu);
        nq[8] = nP[8] + U8 - V8 - W8 + T(1.0 / 36.0) * (even - odd) + nP[8] * (Sb - Sa - csP) -
                T(1.0 / 36.0) * fd(A - B, -cdu, -csu);
    }
}

// One row of the FP32 sub-step: the sums over the row's neighbours on paired
// FP32 instructions (13 moment sums of the f^eq differences, 16 sums of the
// stored f^neq planes) and the closed-form update (see k_fv); sh: the tile's
// staged list, nine planes of hn values.
__device__ __forceinline__ void fv_row_f32(const float *__restrict__ sh, int hn, int own_pos,
                                           const float4 *__restrict__ se, int base, int len, float dt_tau,
                                           int n_ent, float &r1, float &ux, float &uy, float nq[9])
{
    (void)n_ent;
    // own state from the staged list
    float r1P, uPx, uPy, nP[9];
    {
        const int p = HLBM_CHK(own_pos, hn, kSiteStaged);
        r1P = sh[p];
        uPx = sh[hn + p];
        uPy = sh[2 * hn + p];
#pragma unroll
        for (int i = 3; i < 9; i++) nP[i] = sh[i * hn + p];
        neq_complete(nP);
    }
    // own node: no streaming term (g(P) - g(P) = 0), collision weight C_PP = 11/18
    // f^neq part of the sums, over the six stored planes j = 3..8 only:
    //   U_j = sum_k a_k n_j(P_k), V_j = sum_k b_k n_j(P_k), W_j = sum_k cs_k n_j(P_k)
    // (U_4 and V_3 are never needed: c_4x = c_3y = 0); planes 0-2 follow at the
    // end from the same linear constraints that complete f^neq.
    float U3 = 0, U5 = 0, U6 = 0, U7 = 0, U8 = 0, V4 = 0, V5 = 0, V6 = 0, V7 = 0, V8 = 0;
    float W3 = 0, W4 = 0, W5 = 0, W6 = 0, W7 = 0, W8 = 0;
    float Sa = 0, Sb = 0, Dx = 0, Dy = 0, Qxx = 0, Qyy = 0, Qxy = 0, Lx = 0, Ly = 0, Mx = 0, My = 0, Mxxy = 0, Mxyy = 0;
    // the same sums on packed pairs: (U5,U6) (U7,U8) (V5,V6) (V7,V8) (U3,V4)
    // (W3,W4) (W5,W6) (W7,W8) (Sa,Sb) (Dx,Dy) (Qxx,Qyy) (Qxy',Qxy'') (Lx,Ly)
    // (Mx,My) (Mxxy,Mxyy)
    const unsigned long long z = pk2(0.f, 0.f), uP = pk2(uPx, uPy);
    unsigned long long U56 = z, U78 = z, V56 = z, V78 = z, U3V4 = z, W34 = z, W56 = z, W78 = z;
    unsigned long long SS = z, DD = z, QQ = z, QX = z, LL = z, MM = z, MX = z;
    for (int e0 = 0; e0 < len; e0++) {
        float a, b, cs;
        int k;
        unpack(se[HLBM_CHK(base + 32 * e0, n_ent, kSiteEntry)], a, b, cs, k);
        k = HLBM_CHK(k, hn, kSiteStaged);
        const float r1k = sh[k], n3 = sh[3 * hn + k], n4 = sh[4 * hn + k], n5 = sh[5 * hn + k],
                    n6 = sh[6 * hn + k], n7 = sh[7 * hn + k], n8 = sh[8 * hn + k];
        const unsigned long long uk = pk2(sh[hn + k], sh[2 * hn + k]);
        const float drho = r1k - r1P, rhok = 1.f + r1k;
        const unsigned long long ab = pk2(a, b), aa = pk2(a, a), bb = pk2(b, b), cc = pk2(cs, cs);
        const unsigned long long du = sub2(uk, uP), su = add2(uk, uP);   // (dux, duy), (sux, suy)
        const unsigned long long pr = mul2(du, su);                      // (dux sux, duy suy)
        const unsigned long long R = mul2(ab, pk2(rhok, rhok));          // (ra, rb)
        float dux, duy, sux, suy, p0, p1, ra, rb;
        upk2(du, dux, duy);
        upk2(su, sux, suy);
        upk2(pr, p0, p1);
        upk2(R, ra, rb);
        const float dus = p0 + p1, xs = dux * suy + duy * sux;
        SS = add2(SS, ab);
        DD = fma2(ab, pk2(drho, drho), DD);
        QQ = fma2(R, du, QQ);
        QX = fma2(R, pk2(duy, dux), QX);
        LL = fma2(R, pk2(dus, dus), LL);
        MM = fma2(R, pr, MM);
        MX = fma2(R, pk2(xs, xs), fma2(pk2(rb, ra), pr, MX));
        const unsigned long long n34 = pk2(n3, n4), n56 = pk2(n5, n6), n78 = pk2(n7, n8);
        U56 = fma2(aa, n56, U56);
        U78 = fma2(aa, n78, U78);
        V56 = fma2(bb, n56, V56);
        V78 = fma2(bb, n78, V78);
        U3V4 = fma2(ab, n34, U3V4);
        W34 = fma2(cc, n34, W34);
        W56 = fma2(cc, n56, W56);
        W78 = fma2(cc, n78, W78);
    }
    float q0, q1;
    upk2(U56, U5, U6); upk2(U78, U7, U8); upk2(V56, V5, V6); upk2(V78, V7, V8); upk2(U3V4, U3, V4);
    upk2(W34, W3, W4); upk2(W56, W5, W6); upk2(W78, W7, W8);
    upk2(SS, Sa, Sb); upk2(DD, Dx, Dy); upk2(QQ, Qxx, Qyy); upk2(QX, q0, q1); Qxy = q0 + q1;
    upk2(LL, Lx, Ly); upk2(MM, Mx, My); upk2(MX, Mxxy, Mxyy);
    // Update.  With acc_i = sum_k (c_i.(a_k, b_k) - cs_k) f^neq_i(P_k) + w_i eq_i
    // - f^neq_i(P) (c_i.(Sa, Sb) + dt/tau_u C_PP) the increment of population i,
    // its zeroth and first moments need no per-population sum: f^neq carries
    // no mass or momentum and the D2Q9 weights are isotropic to fourth order,
    //   drho = u_P.D + Q_xx + Q_yy
    //   djx  = D_x/3 + u_Px (u_P.D) + 3/2 M_x + 1/2 M_xyy - 1/2 L_x
    //          + sum_k (a_k Pi^neq_xx(P_k) + b_k Pi^neq_xy(P_k)) - (Sa Pi^neq_xx(P) + Sb Pi^neq_xy(P))
    // (djy likewise), with sum_k a_k Pi^neq_xx(P_k) = 2 (U3 + U6 + U7) and so
    // on.  The new f^neq is then needed for the stored planes 3..8 only;
    // opposite diagonals (5, 7) and (6, 8) share the even and odd parts of
    // eq_i and of the f^eq difference.
    const float csP = dt_tau * (11.f / 18.f);
    const float Pxx = nP[1] + nP[3] + nP[5] + nP[6] + nP[7] + nP[8];
    const float Pyy = nP[2] + nP[4] + nP[5] + nP[6] + nP[7] + nP[8];
    const float Pxy = nP[5] - nP[6] + nP[7] - nP[8];
    const float uD = uPx * Dx + uPy * Dy;
    const float drho = uD + Qxx + Qyy;
    const float djx = Dx * (1.f / 3.f) + uPx * uD + 1.5f * Mx + 0.5f * Mxyy - 0.5f * Lx + 2.f * (U3 + U6 + U7) +
                  (V5 - V6 + V7 - V8) - (Sa * Pxx + Sb * Pxy);
    const float djy = Dy * (1.f / 3.f) + uPy * uD + 1.5f * My + 0.5f * Mxxy - 0.5f * Ly + (U5 - U6 + U7 - U8) +
                  2.f * (V4 + V7 + V8) - (Sb * Pyy + Sa * Pxy);
    r1 = r1P + drho;
    const float rho = 1.f + r1, irho = 1.f / rho;
    const float dux = (djx - drho * uPx) * irho, duy = (djy - drho * uPy) * irho;
    ux = uPx + dux;
    uy = uPy + duy;
    const float sx = ux + uPx, sy = uy + uPy;           // u' + u_P
    const float E0 = 1.f - 1.5f * (uPx * uPx + uPy * uPy);
    const float ddot = 1.5f * (dux * sx + duy * sy);  // 3/2 du.(u' + u_P)
    // the same on pairs of directions: (3, 4) mirror each other in x <-> y;
    // (5, 6) and (7, 8) are the two diagonal families' + and - members
    const F2 U = f2(uPx, uPy);
    const F2 E34 = fmaf2(f2(4.5f) * U, U, f2(E0) - f2(3.f) * U);
    const F2 eq34 = f2(3.f) * f2(Qxx, Qyy) + f2(1.5f) * f2(Lx, Ly) - E34 * f2(Dx, Dy) - f2(4.5f) * f2(Mx, My);
    const F2 n34 = f2(nP[3], nP[4]);
    const F2 cdu34 = f2(-dux, -duy), csu34 = f2(-sx, -sy);
    const F2 fd34 = fmaf2(f2(drho), E34,
                          f2(rho) * (fmaf2(f2(4.5f) * cdu34, csu34, f2(3.f) * cdu34) - f2(ddot)));
    const F2 nq34 = n34 - f2(U3, V4) - f2(W3, W4) + fmaf2(n34, f2(Sa - csP, Sb - csP), f2(1.f / 9.f) * (eq34 - fd34));
    const F2 q = f2(uPx + uPy, uPy - uPx);
    const F2 A = fmaf2(f2(4.5f) * q, q, f2(E0)), B = f2(3.f) * q;
    const F2 Pd = f2(Dx + Dy, Dy - Dx);
    const F2 Cq = f2(3.f) * f2(Qxx + Qyy + Qxy, Qxx + Qyy - Qxy);
    const F2 Z = f2(4.5f) * f2(Mx + My + Mxxy + Mxyy, My - Mx + Mxxy - Mxyy) - f2(1.5f) * f2(Lx + Ly, Ly - Lx);
    const F2 odd = fmaf2(A, Pd, Z), even = fmaf2(B, Pd, Cq);
    const F2 cdu = f2(dux + duy, duy - dux), csu = f2(sx + sy, sy - sx);
    const F2 t3 = fmaf2(f2(4.5f) * cdu, csu, f2(3.f) * cdu);  // 3 c.du + 9/2 (c.du)(c.su), + members
    const F2 t3m = fmaf2(f2(4.5f) * cdu, csu, f2(-3.f) * cdu);  // the same for - members
    const F2 fdp = fmaf2(f2(drho), A + B, f2(rho) * (t3 - f2(ddot)));
    const F2 fdm = fmaf2(f2(drho), A - B, f2(rho) * (t3m - f2(ddot)));
    const F2 n56 = f2(nP[5], nP[6]), n78 = f2(nP[7], nP[8]);
    const F2 nq56 = n56 + f2(U5 + V5 - W5, V6 - U6 - W6) - n56 * f2(Sa + Sb + csP, Sb - Sa + csP) +
                    f2(1.f / 36.f) * (even + odd - fdp);
    const F2 nq78 = n78 - f2(U7 + V7 + W7, V8 - U8 + W8) + n78 * f2(Sa + Sb - csP, Sb - Sa - csP) +
                    f2(1.f / 36.f) * (even - odd - fdm);
    float x0, x1;
    upk2(nq34.v, x0, x1); nq[3] = x0; nq[4] = x1;
    upk2(nq56.v, x0, x1); nq[5] = x0; nq[6] = x1;
    upk2(nq78.v, x0, x1); nq[7] = x0; nq[8] = x1;
}

// The end of one row of the sub-step: the wall rule (u = 0) on wall rows, the
// Eq. 5-6 interface state of the next sub-step on ring rows (unless this is
// the last sub-step), and the store of (rho - 1, u, f^neq_3..8).
template <typename T>
__device__ __forceinline__ void fv_finish_row(T *__restrict__ gn, int Np, int r, int n_wall, int ring_start,
                                              int n_ring, const T *__restrict__ Q0, const T *__restrict__ Q1,
                                              T theta_next, T scale5, int star, T r1, T ux, T uy, T nq[9])
{
    if (r < n_wall) {
        ux = T(0);
        uy = T(0);
    } else if (star && r >= ring_start) {
        int q_ = r - ring_start;
        T a = T(1) - theta_next;
        r1 = a * Q0[q_] + theta_next * Q1[q_] - T(1);
        ux = a * Q0[size_t(n_ring) + q_] + theta_next * Q1[size_t(n_ring) + q_];
        uy = a * Q0[size_t(2) * n_ring + q_] + theta_next * Q1[size_t(2) * n_ring + q_];
#pragma unroll
        for (int i = 3; i < 9; i++)
            nq[i] = scale5 * (a * Q0[size_t(3 + i) * n_ring + q_] + theta_next * Q1[size_t(3 + i) * n_ring + q_]);
    }
    gn[r] = r1;
    gn[size_t(Np) + r] = ux;
    gn[size_t(2) * Np + r] = uy;
#pragma unroll
    for (int i = 3; i < 9; i++) gn[size_t(i) * Np + r] = nq[i];
}

// ROWS: rows per tile (= threads per block); MINB: blocks per SM the
// register allocation is bounded for (1: unbounded).  The FP32 kernel is
// built for 7 and 8 blocks of kTileRows rows and for 3 and 4 blocks of
// kTileRowsWide rows, and each context keeps the fastest for its mesh
// (fv_autotune); FP64 is built unbounded for kTileRows rows.
template <typename T, int MINB, int ROWS>
__global__ void __launch_bounds__(ROWS, MINB) k_fv(const T *__restrict__ g, T *__restrict__ gn, int Np, int n,
                                                   const int *__restrict__ slice_ptr,
                                                   const int *__restrict__ slice_len,
                                                   const typename Ent<T>::type *__restrict__ ent, int max_tile_ent,
                                                   const int *__restrict__ halo_ptr,
                                                   const int *__restrict__ halo_nodes, T dt_tau,
                                                   int n_wall, int ring_start, int n_ring,
                                                   const T *__restrict__ Q0, const T *__restrict__ Q1, T theta_next,
                                                   T scale5, int star, int *flag, int pf_ahead)
{
    using E = typename Ent<T>::type;
    extern __shared__ __align__(16) unsigned char fv_smem[];
    // [0, 16): two mbarriers (entries; the tile's own states); [16, ...): the
    // tile's entries; then the staged states, nine planes of stride hs
    const uint32_t bar_e = uint32_t(__cvta_generic_to_shared(fv_smem)), bar_s = bar_e + 8u;
    const E *se = reinterpret_cast<const E *>(fv_smem + 16);
    T *sh = reinterpret_cast<T *>(fv_smem + 16 + size_t(max_tile_ent) * sizeof(E));
    const int t = blockIdx.x;
    const int e_begin = slice_ptr[(ROWS / 32) * t];
#ifdef HLBM_DEBUG
    const int n_ent = slice_ptr[(ROWS / 32) * (t + 1)] - e_begin;  // entries staged for this tile
#endif
    const int h0 = halo_ptr[t], hn = halo_ptr[t + 1] - h0, hs = (hn + 3) & ~3;
    const int r0 = t * ROWS;
    if (threadIdx.x == 0) {
        const uint32_t bytes =
            uint32_t(HLBM_CHK(slice_ptr[(ROWS / 32) * (t + 1)] - e_begin, max_tile_ent + 1, kSiteEntry)) * uint32_t(sizeof(E));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_e) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("{\n\t.reg .b64 st;\n\t"
                     "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar_e),
                     "r"(bytes)
                     : "memory");
        if (bytes > 0)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             bar_e + 16u),
                         "l"(ent + e_begin), "r"(bytes), "r"(bar_e)
                         : "memory");
    }
    // Let the next sub-step's blocks start as soon as SM slots free up; they
    // only read constant operator data until their griddepcontrol.wait.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int r = r0 + threadIdx.x;
    const int rr = r < n ? r : n - 1;
    const int sl = rr >> 5;
    const int base = slice_ptr[sl] - e_begin + (rr & 31), len = slice_len[sl];
    // the staged list: the tile's own 128 rows (device rows r0 .. r0 + 127, a
    // run of every plane, copied in bulk), then the other nodes its rows
    // touch (gathered)
    int hidx[kFvHaloRegs];
#pragma unroll
    for (int j = 0; j < kFvHaloRegs; j++) {
        const int h = ROWS + threadIdx.x + j * ROWS;
        hidx[j] = h < hn ? HLBM_CHK(halo_nodes[h0 + h], Np, kSiteMesh) : 0;
    }
    // The tile that will start about when this one ends (pf_ahead = the
    // resident blocks of this launch; blocks start in index order): its
    // operator entries and, once the state is ready, its states are
    // prefetched into L2, so that its copies find them there.
    const int tp = pf_ahead > 0 ? t + pf_ahead : int(gridDim.x);
    int pidx[kFvPrefetchRegs], hpn = 0;
    if (tp < int(gridDim.x)) {
        const int hp0 = halo_ptr[tp];
        hpn = halo_ptr[tp + 1] - hp0;
#pragma unroll
        for (int j = 0; j < kFvPrefetchRegs; j++) {
            const int h = ROWS + threadIdx.x + j * ROWS;
            pidx[j] = h < hpn ? HLBM_CHK(halo_nodes[hp0 + h], Np, kSiteMesh) : 0;
        }
        if (threadIdx.x == 0) {
            const int ep = slice_ptr[(ROWS / 32) * tp];
            const uint32_t pbytes = uint32_t(slice_ptr[(ROWS / 32) * (tp + 1)] - ep) * uint32_t(sizeof(E));
            if (pbytes > 0)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(ent + ep), "r"(pbytes) : "memory");
        }
    }
    // wait until the previous sub-step (which wrote g) has completed
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (threadIdx.x == 0) {
        constexpr uint32_t run = uint32_t(ROWS * sizeof(T));  // one plane's run of own rows
        asm volatile("{\n\t.reg .b64 st;\n\t"
                     "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar_s),
                     "r"(9u * run)
                     : "memory");
        const uint32_t dst0 = uint32_t(__cvta_generic_to_shared(sh));
#pragma unroll
        for (int i = 0; i < 9; i++)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             dst0 + uint32_t(i * hs) * uint32_t(sizeof(T))),
                         "l"(g + size_t(i) * Np + HLBM_CHK(r0, Np - ROWS + 1, kSiteMesh)), "r"(run), "r"(bar_s)
                         : "memory");
        if (tp < int(gridDim.x)) {
#pragma unroll
            for (int i = 0; i < 9; i++)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g + size_t(i) * Np + size_t(tp) * ROWS),
                             "r"(run)
                             : "memory");
        }
    }
#pragma unroll
    for (int j = 0; j < kFvHaloRegs; j++) {
        const int h = ROWS + threadIdx.x + j * ROWS;
        if (h < hn) {
#pragma unroll
            for (int i = 0; i < 9; i++) sh[i * hs + h] = g[size_t(i) * Np + hidx[j]];
        }
    }
    for (int h = ROWS * (1 + kFvHaloRegs) + threadIdx.x; h < hn; h += ROWS) {
        const int node = HLBM_CHK(halo_nodes[h0 + h], Np, kSiteMesh);
#pragma unroll
        for (int i = 0; i < 9; i++) sh[i * hs + h] = g[size_t(i) * Np + node];
    }
#pragma unroll
    for (int j = 0; j < kFvPrefetchRegs; j++) {
        if (ROWS + threadIdx.x + j * ROWS < hpn) {
#pragma unroll
            for (int i = 0; i < 9; i++)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(g + size_t(i) * Np + pidx[j]) : "memory");
        }
    }
    __syncthreads();
    if (!mbar_wait(bar_e, 0) || !mbar_wait(bar_s, 0)) {
        // a bulk copy did not arrive: report, give both copies one more
        // bounded wait (they target this block's shared memory) and leave
        if (threadIdx.x == 0) atomicOr(flag, kFlagTimeout);
        mbar_wait(bar_e, 0);
        mbar_wait(bar_s, 0);
        return;
    }
    if (r >= n) return;
    T r1, ux, uy, nq[9];
#ifdef HLBM_DEBUG
    const int n_ent_chk = n_ent;
#else
    const int n_ent_chk = 0;
#endif
    if constexpr (sizeof(T) == 4)
        fv_row_f32(sh, hs, int(threadIdx.x), se, base, len, dt_tau, n_ent_chk, r1, ux, uy, nq);
    else
        fv_row_f64<T>(sh, hs, int(threadIdx.x), se, base, len, dt_tau, n_ent_chk, r1, ux, uy, nq);
    fv_finish_row<T>(gn, Np, r, n_wall, ring_start, n_ring, Q0, Q1, theta_next, scale5, star, r1, ux, uy, nq);
}

// FP32 -> FP64 copy (the adjoint's records of an FP32 forward).
__global__ void k_widen(const float *__restrict__ a, double *__restrict__ b, size_t n)
{
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        b[i] = double(a[i]);
}

// Odd-even filter of the mesh state, once per finest step after the Eq. 3
// sub-steps (an addition to the paper's method, off unless the context is
// created with fv_filter = sigma > 0): with the graph Laplacian of the Eq. 3
// collision weights, (L g)_i(P) = sum_{k != P} C_Pk [g_i(P_k) - g_i(P)],
//   g <- g - sigma L d,  d = L g on fluid rows, 0 on wall and ring rows,
// on the fluid rows; wall and ring rows keep their state (at a boundary row L
// is a one-sided first-order difference).  C_Pk is read back from the
// operator entries (stored as dt/tau_u C_Pk: C_Pk = entry * c_scale,
// c_scale = tau_u / dt); A_P C_Pk is symmetric.  Two passes, one
// thread per row, neighbours gathered from global memory (L2):
// k_fv_lap writes L g ([9][Np], differences g(P_k) - g(P) formed as in the
// sub-step: f^eq through moment differences, f^neq directly), k_fv_bilap
// applies -sigma L to it and updates the (rho, u, f^neq) state.
template <typename T>
__global__ void __launch_bounds__(128) k_fv_lap(const T *__restrict__ g, T *__restrict__ lap, int Np, int n,
                                                 const int *__restrict__ slice_ptr, const int *__restrict__ slice_len,
                                                 const typename Ent<T>::type *__restrict__ ent,
                                                 const int *__restrict__ halo_ptr, const int *__restrict__ halo_nodes,
                                                 int rows, T c_scale, int n_wall, int ring_start)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    if (r < n_wall || r >= ring_start) {
#pragma unroll
        for (int i = 0; i < 9; i++) lap[size_t(i) * Np + r] = T(0);
        return;
    }
    T r1P, uPx, uPy, nP[9];
    load_mesh(g, Np, r, r1P, uPx, uPy, nP);
    T E[9], acc[9];
#pragma unroll
    for (int i = 0; i < 9; i++) {
        E[i] = Efun<T>(i, uPx, uPy);
        acc[i] = T(0);
    }
    const int sl = r >> 5, base = slice_ptr[sl] + (r & 31), len = slice_len[sl];
    const int h0 = halo_ptr[r / rows];
    for (int e = 0; e < len; e++) {
        T a, b, cs;
        int col;
        unpack(ent[base + 32 * e], a, b, cs, col);
        if (cs == T(0)) continue;  // padding entry
        const T w = cs * c_scale;
        const int k = HLBM_CHK(halo_nodes[h0 + col], Np, kSiteMesh);
        T r1k, ukx, uky, nk[9];
        load_mesh(g, Np, k, r1k, ukx, uky, nk);
        const T drho = r1k - r1P, rhok = T(1) + r1k;
        const T dux = ukx - uPx, duy = uky - uPy, sux = ukx + uPx, suy = uky + uPy;
#pragma unroll
        for (int i = 0; i < 9; i++) acc[i] += w * (feq_diff<T>(i, E[i], drho, rhok, dux, duy, sux, suy) + nk[i] - nP[i]);
    }
#pragma unroll
    for (int i = 0; i < 9; i++) lap[size_t(i) * Np + r] = acc[i];
}

template <typename T>
__global__ void __launch_bounds__(128) k_fv_bilap(const T *__restrict__ g, const T *__restrict__ lap,
                                                   T *__restrict__ gn, int Np, int n,
                                                   const int *__restrict__ slice_ptr, const int *__restrict__ slice_len,
                                                   const typename Ent<T>::type *__restrict__ ent,
                                                   const int *__restrict__ halo_ptr,
                                                   const int *__restrict__ halo_nodes, int rows, T c_scale, T sigma,
                                                   int n_wall, int ring_start)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    if (r < n_wall || r >= ring_start) {  // boundary rows: unchanged
#pragma unroll
        for (int i = 0; i < 9; i++) gn[size_t(i) * Np + r] = g[size_t(i) * Np + r];
        return;
    }
    T dP[9], acc[9];
#pragma unroll
    for (int i = 0; i < 9; i++) {
        dP[i] = lap[size_t(i) * Np + r];
        acc[i] = T(0);
    }
    const int sl = r >> 5, base = slice_ptr[sl] + (r & 31), len = slice_len[sl];
    const int h0 = halo_ptr[r / rows];
    for (int e = 0; e < len; e++) {
        T a, b, cs;
        int col;
        unpack(ent[base + 32 * e], a, b, cs, col);
        if (cs == T(0)) continue;
        const T w = cs * c_scale;
        const int k = HLBM_CHK(halo_nodes[h0 + col], Np, kSiteMesh);
#pragma unroll
        for (int i = 0; i < 9; i++) acc[i] += w * (lap[size_t(i) * Np + k] - dP[i]);
    }
    T r1P, uPx, uPy, nP[9];
    load_mesh(g, Np, r, r1P, uPx, uPy, nP);
    T drho = 0, djx = 0, djy = 0;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        acc[i] *= -sigma;
        drho += acc[i];
        djx += T(cx(i)) * acc[i];
        djy += T(cy(i)) * acc[i];
    }
    const T rho = T(1) + r1P + drho;
    T ux = uPx + (djx - drho * uPx) / rho, uy = uPy + (djy - drho * uPy) / rho;
    const T dux = ux - uPx, duy = uy - uPy, sux = ux + uPx, suy = uy + uPy;
    T nq[9];
#pragma unroll
    for (int i = 0; i < 9; i++)
        nq[i] = nP[i] + acc[i] - feq_diff<T>(i, Efun<T>(i, uPx, uPy), drho, rho, dux, duy, sux, suy);
    gn[r] = r1P + drho;
    gn[size_t(Np) + r] = ux;
    gn[size_t(2) * Np + r] = uy;
#pragma unroll
    for (int i = 3; i < 9; i++) gn[size_t(i) * Np + r] = nq[i];
}

// Eq. 10-11: force on the body from nodal pressure and stress at the wall,
// traction -(p - p0) n - Pi^neq . n with p = rho / 3, edge values the mean of
// the two end nodes.  Two passes with a fixed summation order (deterministic):
// k_forces_partial writes one FP64 (F_x, F_y) partial per block of wall
// edges, k_forces_final adds the partials in block order and records
// (C_D, C_L) in the ring buffer.
constexpr int kForceThreads = 128;

template <typename T>
__device__ __forceinline__ void edge_force(const T *g, int Np, int a, int b, double nx, double ny, double &fx,
                                           double &fy)
{
    double p = 0, pxx = 0, pxy = 0, pyy = 0;
    for (int s = 0; s < 2; s++) {
        int k = s ? b : a;
        T q[12];
        mesh_q(g, Np, k, q);
        p += 0.5 * double(q[0]) / 3.0;
#pragma unroll
        for (int i = 0; i < 9; i++) {
            double nq = double(q[3 + i]);
            pxx += 0.5 * cx(i) * cx(i) * nq;
            pxy += 0.5 * cx(i) * cy(i) * nq;
            pyy += 0.5 * cy(i) * cy(i) * nq;
        }
    }
    double pm = p - 1.0 / 3.0;
    fx = -pm * nx - (pxx * nx + pxy * ny);
    fy = -pm * ny - (pxy * nx + pyy * ny);
}

__device__ __forceinline__ void block_sum2(double &fx, double &fy)
{
    __shared__ double sx[32], sy[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_down_sync(0xffffffffu, fx, o);
        fy += __shfl_down_sync(0xffffffffu, fy, o);
    }
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sx[warp] = fx; sy[warp] = fy; }
    __syncthreads();
    if (warp == 0) {
        int nw = (blockDim.x + 31) >> 5;
        fx = lane < nw ? sx[lane] : 0.0;
        fy = lane < nw ? sy[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fx += __shfl_down_sync(0xffffffffu, fx, o);
            fy += __shfl_down_sync(0xffffffffu, fy, o);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kForceThreads) k_forces_partial(const T *g, int Np, const int *wea, const int *web,
                                                                  const double *wn, int n_edges, double *partial)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    double fx = 0.0, fy = 0.0;
    if (e < n_edges) edge_force(g, Np, wea[e], web[e], wn[2 * e], wn[2 * e + 1], fx, fy);
    block_sum2(fx, fy);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = fx;
        partial[2 * blockIdx.x + 1] = fy;
    }
}
// Eq. 12-13 at the wall rows (device rows 0 .. n_wall-1): C_p = (rho - 1) / 3 / q
// and the viscous traction -Pi^neq n split along the unit normal n and the
// downstream tangent s (C_n, C_f), added to FP64 sums [3][n_wall].
template <typename T>
__global__ void k_wall_stats(const T *g, int Np, int n_wall, const double *ns, double *acc, double inv_q)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_wall) return;
    T q[12];
    mesh_q(g, Np, r, q);
    double pxx = 0, pxy = 0, pyy = 0;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const double nq = double(q[3 + i]);
        pxx += cx(i) * cx(i) * nq;
        pxy += cx(i) * cy(i) * nq;
        pyy += cy(i) * cy(i) * nq;
    }
    const double nx = ns[4 * r], ny = ns[4 * r + 1], sx = ns[4 * r + 2], sy = ns[4 * r + 3];
    const double tx = -(pxx * nx + pxy * ny), ty = -(pxy * nx + pyy * ny);
    acc[r] += (double(q[0]) - 1.0) / 3.0 * inv_q;
    acc[size_t(n_wall) + r] += (tx * sx + ty * sy) * inv_q;
    acc[size_t(2) * n_wall + r] += (tx * nx + ty * ny) * inv_q;
}


__global__ void __launch_bounds__(kForceThreads) k_forces_final(const double *partial, int n_part, double qdyn,
                                                                double *buf, int *counter, int cap, int *flag)
{
    double fx = 0.0, fy = 0.0;
    for (int b = threadIdx.x; b < n_part; b += blockDim.x) {
        fx += partial[2 * b];
        fy += partial[2 * b + 1];
    }
    block_sum2(fx, fy);
    if (threadIdx.x == 0) {
        int c = *counter;
        buf[2 * (c % cap)] = fx / qdyn;
        buf[2 * (c % cap) + 1] = fy / qdyn;
        *counter = c + 1;
        if (!(fx == fx) || !(fy == fy)) *flag = 1;
    }
}

// Density, velocity (and optionally populations) of a level in FP64, x fastest;
// NaN on nodes that are not computed (the hole and the coarse nodes over it).
template <typename T, typename S, int P>
__global__ void k_fields_level(const S *f, int nx, int ny, int pitch, size_t stride, const int *hx0, const int *hx1,
                               double *rho, double *ux, double *uy, double *pop, LatShift sh)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    size_t o = size_t(y) * nx + x;
    if (hx0 && x >= hx0[y] && x < hx1[y]) {
        if (rho) { rho[o] = NAN; ux[o] = NAN; uy[o] = NAN; }
        if (pop)
            for (int i = 0; i < 9; i++) pop[9 * o + i] = NAN;
        return;
    }
    T d[9];
    load_state<T, S, P>(f, node(x, y, pitch), pitch, stride, d, sh);
    if (rho) {
        double dd[9];
        for (int i = 0; i < 9; i++) dd[i] = double(d[i]);
        double r, u, v;
        moments(dd, r, u, v);
        rho[o] = r; ux[o] = u; uy[o] = v;
    }
    if (pop)
        for (int i = 0; i < 9; i++) pop[9 * o + i] = double(d[i]) + wq<double>(i);
}

// Total mass of level 0 (it spans the whole domain; refined levels restrict
// into it), FP64 in every precision, deterministic: one block per row sums
// sum_i (f_i - w_i) over the row's computed nodes in a fixed order, then one
// block adds the rows in order.  The host adds the node count.
constexpr int kMassThreads = 256;

template <typename T, typename S, int P>
__global__ void __launch_bounds__(kMassThreads) k_mass_rows(const S *f, int nx, int pitch, size_t stride,
                                                            const int *hx0, const int *hx1, double *row_sum,
                                                            LatShift sh)
{
    const int y = blockIdx.x;
    double acc = 0.0;
    for (int x = threadIdx.x; x < nx; x += kMassThreads) {
        if (hx0 && x >= hx0[y] && x < hx1[y]) continue;
        T d[9];
        load_state<T, S, P>(f, node(x, y, pitch), pitch, stride, d, sh);
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < 9; i++) s += double(d[i]);
        acc += s;
    }
    __shared__ double red[kMassThreads];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kMassThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) row_sum[y] = red[0];
}

__global__ void __launch_bounds__(kMassThreads) k_mass_total(const double *row_sum, int ny, double *out)
{
    __shared__ double red[kMassThreads];
    double acc = 0.0;
    for (int y = threadIdx.x; y < ny; y += kMassThreads) acc += row_sum[y];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kMassThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

template <typename T>
__global__ void k_fields_mesh(const T *g, int Np, const int *inv, int n, double *rho, double *ux, double *uy,
                              double *pop)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int k = inv[p];
    T q[12];
    mesh_q(g, Np, k, q);
    if (rho) {
        rho[p] = double(q[0]); ux[p] = double(q[1]); uy[p] = double(q[2]);
    }
    if (pop)
        for (int i = 0; i < 9; i++)
            pop[9 * size_t(p) + i] = wq<double>(i) + deq<double>(i, double(q[0]), double(q[1]), double(q[2])) + double(q[3 + i]);
}

inline unsigned cdiv(long a, long b) { return unsigned((a + b - 1) / b); }

}  // namespace

// ------------------------------------------------------------ launchers ----
// T: arithmetic type; S: lattice storage type (T, or __half for FP16S).
template <typename T, typename S>
void launch_init_level(const DevCtx &C, int c, unsigned long long seed, double perturb, cudaStream_t s)
{
    const DevLevel &l = C.lv[c];
    dim3 grid(cdiv(l.nx + 2, 128), l.ny + 2);
    k_init_level<T, S><<<grid, 128, 0, s>>>((S *)l.f, l.nx, l.ny, l.pitch, l.stride, l.hx0, l.hx1, seed, c, perturb,
                                            C.u0, C.shift);
}

template <typename T, typename S> void launch_collide(const DevCtx &C, int c, cudaStream_t s)
{
    const DevLevel &l = C.lv[c];
    dim3 grid(cdiv(l.nx, kCollideThreads * kCollideNodes), l.ny);
    T omega = T(1.0 / l.tau);
    if (l.parity == 0)
        k_collide<T, S, 0><<<grid, kCollideThreads, 0, s>>>((S *)l.f, l.nx, l.ny, l.pitch, l.stride, omega, l.hx0,
                                                            l.hx1, C.shift);
    else
        k_collide<T, S, 1><<<grid, kCollideThreads, 0, s>>>((S *)l.f, l.nx, l.ny, l.pitch, l.stride, omega, l.hx0,
                                                            l.hx1, C.shift);
}

template <typename T, typename S> void launch_outer_bc(const DevCtx &C, cudaStream_t s)
{
    const DevLevel &l = C.lv[0];
    int nper = 2 * l.nx + 2 * (l.ny - 2);
    if (l.parity == 0)
        k_outer_bc<T, S, 0><<<cdiv(nper, 128), 128, 0, s>>>((S *)l.f, l.nx, l.ny, l.pitch, l.stride, T(C.u0), C.shift);
    else
        k_outer_bc<T, S, 1><<<cdiv(nper, 128), 128, 0, s>>>((S *)l.f, l.nx, l.ny, l.pitch, l.stride, T(C.u0), C.shift);
}

template <typename T, typename S> void launch_snapshot(const DevCtx &C, int c, bool into_b, cudaStream_t s)
{
    const DevLevel &l = C.lv[c];
    T *dst = (T *)(into_b ? l.snapB : l.snapA);
    if (l.parity == 0)
        k_snapshot<T, S, 0><<<cdiv(l.band_n, 128), 128, 0, s>>>((const S *)l.f, l.pitch, l.stride, l.cox, l.coy, l.cmx,
                                                                 l.cmy, dst, l.band_n, C.shift);
    else
        k_snapshot<T, S, 1><<<cdiv(l.band_n, 128), 128, 0, s>>>((const S *)l.f, l.pitch, l.stride, l.cox, l.coy, l.cmx,
                                                                 l.cmy, dst, l.band_n, C.shift);
}

template <typename T, typename S> void launch_prolong(const DevCtx &C, int cf, double theta, cudaStream_t s)
{
    const DevLevel &p = C.lv[cf - 1], &l = C.lv[cf];
    int nper = 2 * l.nx + 2 * (l.ny - 2);
    T scale = T(l.tau / (2.0 * p.tau));
    if (l.parity == 0)
        k_prolong<T, S, 0><<<cdiv(nper, 128), 128, 0, s>>>((S *)l.f, l.nx, l.ny, l.pitch, l.stride, (const T *)p.snapA,
                                                            (const T *)p.snapB, p.band_n, p.cox, p.coy, p.cmx, p.cmy,
                                                            T(theta), scale, C.shift);
    else
        k_prolong<T, S, 1><<<cdiv(nper, 128), 128, 0, s>>>((S *)l.f, l.nx, l.ny, l.pitch, l.stride, (const T *)p.snapA,
                                                            (const T *)p.snapB, p.band_n, p.cox, p.coy, p.cmx, p.cmy,
                                                            T(theta), scale, C.shift);
}

template <typename T, typename S> void launch_restrict(const DevCtx &C, int cc, cudaStream_t s)
{
    const DevLevel &p = C.lv[cc], &l = C.lv[cc + 1];
    if (p.cmx < 2 || p.cmy < 2) return;
    dim3 grid(cdiv(p.cmx - 1, 128), p.cmy - 1);
    T scale = T(2.0 * p.tau / l.tau);
#define HLBM_RESTRICT(PC, PF)                                                                                        \
    k_restrict<T, S, PC, PF><<<grid, 128, 0, s>>>((S *)p.f, p.pitch, p.stride, (const S *)l.f, l.pitch, l.stride,     \
                                                  p.cox, p.coy, p.cmx, p.cmy, scale, p.hx0, p.hx1, C.shift)
    if (p.parity == 0 && l.parity == 0) HLBM_RESTRICT(0, 0);
    else if (p.parity == 0) HLBM_RESTRICT(0, 1);
    else if (l.parity == 0) HLBM_RESTRICT(1, 0);
    else HLBM_RESTRICT(1, 1);
#undef HLBM_RESTRICT
}

template <typename T, typename S> void launch_ring_interp(const DevCtx &C, bool q1_and_star, cudaStream_t s)
{
    const DevLevel &l = C.lv[C.L - 1];
    const DevMesh &m = C.m;
    if (m.n_ring == 0) return;
    T scale5 = T(1.0 - 1.0 / (2.0 * l.tau));
    T *Q = (T *)(q1_and_star ? m.Q1 : m.Q0);
    T *g = (T *)m.g[m.gcur];
    int star = q1_and_star ? 1 : 0;
    if (l.parity == 0)
        k_ring_interp<T, S, 0><<<cdiv(16L * m.n_ring, 128), 128, 0, s>>>(
            (const S *)l.f, l.pitch, l.stride, m.ring_don, (const T *)m.ring_w, m.n_ring, Q, (const T *)m.Q0, g, m.Np,
            m.ring_start, scale5, star, C.shift);
    else
        k_ring_interp<T, S, 1><<<cdiv(16L * m.n_ring, 128), 128, 0, s>>>(
            (const S *)l.f, l.pitch, l.stride, m.ring_don, (const T *)m.ring_w, m.n_ring, Q, (const T *)m.Q0, g, m.Np,
            m.ring_start, scale5, star, C.shift);
}

template <typename T, typename S> void launch_hole_interp(const DevCtx &C, cudaStream_t s)
{
    const DevLevel &l = C.lv[C.L - 1];
    const DevMesh &m = C.m;
    if (m.n_is == 0) return;
    T scale4 = T(2.0 * (l.tau - 1.0) / (2.0 * l.tau - 1.0));
    if (l.parity == 0)
        k_hole_interp<T, S, 0><<<cdiv(8L * m.n_is, 128), 128, 0, s>>>((S *)l.f, l.pitch, l.stride, m.is_n, m.is_don,
                                                                      (const T *)m.is_w, m.n_is, (const T *)m.g[m.gcur],
                                                                      m.Np, scale4, C.shift);
    else
        k_hole_interp<T, S, 1><<<cdiv(8L * m.n_is, 128), 128, 0, s>>>((S *)l.f, l.pitch, l.stride, m.is_n, m.is_don,
                                                                      (const T *)m.is_w, m.n_is, (const T *)m.g[m.gcur],
                                                                      m.Np, scale4, C.shift);
}

template <typename T, typename S> void launch_fv(const DevCtx &C, int msub, cudaStream_t s)
{
    const DevMesh &m = C.m;
    const FvTiles &tl = m.tl;
    const DevLevel &l = C.lv[C.L - 1];
    T dt_tau = T(C.dt_u / C.tau_u);
    T scale5 = T(1.0 - 1.0 / (2.0 * l.tau));
    int star = msub < C.n_sub - 1 ? 1 : 0;
    T theta_next = T(double(msub + 1) / double(C.n_sub));
    // programmatic dependent launch: the sub-step may begin while the previous
    // kernel on the stream drains (it waits for it before reading the state)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(tl.n_tiles));
    cfg.blockDim = dim3(unsigned(tl.rows));
    cfg.dynamicSmemBytes = tl.smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // variants: 1, 2 bounded for the lower and the higher block count per SM;
    // 3, 4 the same with the L2 prefetch of a later tile (FP64: one
    // unbounded kernel)
    const int v = m.fv_variant, bound = (v == 2 || v == 4) ? 2 : 1;
    const int pf = v >= 3 ? tl.pf_ahead[bound] : 0;
    auto go = [&](auto kern) {
        cudaLaunchKernelEx(&cfg, kern, (const T *)m.g[m.gcur], (T *)m.g[m.gcur ^ 1], m.Np, m.n,
                           (const int *)m.slice_ptr, (const int *)m.slice_len, (const typename Ent<T>::type *)tl.ent,
                           tl.max_tile_ent, (const int *)tl.halo_ptr, (const int *)tl.halo_nodes,
                           dt_tau, m.n_wall, m.ring_start, m.n_ring, (const T *)m.Q0,
                           (const T *)m.Q1, theta_next, scale5, star, C.flag, pf);
    };
    if constexpr (sizeof(T) == 4) {
        if (tl.rows == kTileRowsWide) {
            if (bound == 2) go(k_fv<T, 4, kTileRowsWide>);
            else go(k_fv<T, 3, kTileRowsWide>);
        } else {
            if (bound == 2) go(k_fv<T, 8, kTileRows>);
            else go(k_fv<T, 7, kTileRows>);
        }
    } else {
        go(k_fv<T, 1, kTileRows>);
    }
}

template <typename T, typename S> void launch_fv_filter(const DevCtx &C, cudaStream_t s)
{
    const DevMesh &m = C.m;
    if (m.n == 0 || !(C.fv_filter > 0.0) || !m.lap) return;
    const T c_scale = T(C.tau_u / C.dt_u);
    const unsigned nb = cdiv(m.n, 128);
    using E = typename Ent<T>::type;
    const FvTiles &tl = m.tl;
    k_fv_lap<T><<<nb, 128, 0, s>>>((const T *)m.g[m.gcur], (T *)m.lap, m.Np, m.n, (const int *)m.slice_ptr,
                                   (const int *)m.slice_len, (const E *)tl.ent, (const int *)tl.halo_ptr,
                                   (const int *)tl.halo_nodes, tl.rows, c_scale, m.n_wall, m.ring_start);
    k_fv_bilap<T><<<nb, 128, 0, s>>>((const T *)m.g[m.gcur], (const T *)m.lap, (T *)m.g[m.gcur ^ 1], m.Np, m.n,
                                     (const int *)m.slice_ptr, (const int *)m.slice_len, (const E *)tl.ent,
                                     (const int *)tl.halo_ptr, (const int *)tl.halo_nodes, tl.rows, c_scale,
                                     T(C.fv_filter), m.n_wall, m.ring_start);
}

void launch_widen(const float *a, double *b, size_t n, cudaStream_t s)
{
    if (n == 0) return;
    const unsigned nb = unsigned(std::min<size_t>((n + 255) / 256, 152 * 16));
    k_widen<<<nb, 256, 0, s>>>(a, b, n);
}

// Autotuner of the sub-step kernel (FP32): on each tiling built (kTileRows
// rows per tile and, if the set-up built it, kTileRowsWide) times each
// variant on this mesh (reps launches reading the current state buffer and
// writing the other one, which the next sub-step overwrites, so the state is
// unchanged): 1, 2 registers bounded for the lower and the higher block count
// per SM (7, 8 blocks of 128 rows; 3, 4 blocks of 256), 3, 4 the same with the
// L2 prefetch of a later tile's entries and halo states.  us[0..3] and
// us[4..7] receive the mean launch times of the two tilings.  Leaves the
// fastest in m.tl and m.fv_variant (the other tiling in m.tl_alt) and returns
// it as 1..8.  Variants of one tiling execute the same arithmetic; the two
// tilings order each row's entries for their own shared-memory banks.
template <typename T, typename S> int fv_autotune(DevCtx &C, cudaStream_t s, double us[8])
{
    for (int k = 0; k < 8; k++) us[k] = 0.0;
    if constexpr (sizeof(T) != 4) {
        return 1;
    } else {
        DevMesh &m = C.m;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            if (e0) cudaEventDestroy(e0);
            return 1;
        }
        const int reps = 20;
        int best = 0;  // 0..7
        for (int w = 0; w < 2; w++) {
            if (w == 1) {
                if (m.tl_alt.rows == 0) break;
                std::swap(m.tl, m.tl_alt);
            }
            for (int v = 1; v <= 4; v++) {
                m.fv_variant = v;
                for (int k = 0; k < 3; k++) launch_fv<T, S>(C, 0, s);
                cudaEventRecord(e0, s);
                for (int k = 0; k < reps; k++) launch_fv<T, S>(C, 0, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                us[4 * w + v - 1] = 1e3 * double(ms) / reps;
                if (us[4 * w + v - 1] < us[best]) best = 4 * w + v - 1;
            }
        }
        // m.tl is the tiling timed last: keep the best one there
        const bool wide_last = m.tl.rows == kTileRowsWide;
        const bool want_wide = best >= 4;
        if (wide_last != want_wide && m.tl_alt.rows != 0) std::swap(m.tl, m.tl_alt);
        m.fv_variant = best % 4 + 1;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return best + 1;
    }
}

// Raises the dynamic shared-memory limit of the tiling's kernels to the
// device's opt-in maximum when the tiling needs more than the default (a
// per-kernel setting shared by every context of the process, so it is never
// lowered).
template <typename T, typename S> void configure_fv(const FvTiles &tl)
{
    if (tl.smem_bytes <= 48 * 1024) return;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if constexpr (sizeof(T) == 4) {
        if (tl.rows == kTileRowsWide) {
            cudaFuncSetAttribute(k_fv<T, 3, kTileRowsWide>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
            cudaFuncSetAttribute(k_fv<T, 4, kTileRowsWide>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        } else {
            cudaFuncSetAttribute(k_fv<T, 7, kTileRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
            cudaFuncSetAttribute(k_fv<T, 8, kTileRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        }
    } else {
        cudaFuncSetAttribute(k_fv<T, 1, kTileRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    }
}

template <typename T, typename S> void configure_fv_prefetch(FvTiles &tl)
{
    int dev = 0, sms = 0;
    for (int v = 0; v < 3; v++) tl.pf_ahead[v] = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    auto resident = [&](auto kern) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tl.rows, tl.smem_bytes) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return per_sm * sms;
    };
    if constexpr (sizeof(T) == 4) {
        if (tl.rows == kTileRowsWide) {
            tl.pf_ahead[1] = resident(k_fv<T, 3, kTileRowsWide>);
            tl.pf_ahead[2] = resident(k_fv<T, 4, kTileRowsWide>);
        } else {
            tl.pf_ahead[1] = resident(k_fv<T, 7, kTileRows>);
            tl.pf_ahead[2] = resident(k_fv<T, 8, kTileRows>);
        }
    } else {
        tl.pf_ahead[1] = resident(k_fv<T, 1, kTileRows>);
    }
}

bool debug_bounds(unsigned int out[2])
{
#ifdef HLBM_DEBUG
    if (cudaMemcpyFromSymbol(out, d_bounds, 2 * sizeof(unsigned int)) == cudaSuccess) return true;
#endif
    out[0] = out[1] = 0;
    return false;
}

template <typename T, typename S> void launch_forces(const DevCtx &C, cudaStream_t s)
{
    const DevMesh &m = C.m;
    int nb = std::max(1, int(cdiv(m.n_edges, kForceThreads)));
    k_forces_partial<T><<<nb, kForceThreads, 0, s>>>((const T *)m.g[m.gcur], m.Np, m.wea, m.web, m.wn, m.n_edges,
                                                     C.force_partial);
    k_forces_final<<<1, kForceThreads, 0, s>>>(C.force_partial, nb, C.qdyn, C.force_buf, C.force_counter,
                                               C.force_cap, C.flag);
}

template <typename T, typename S> void launch_wall_stats(const DevCtx &C, cudaStream_t s)
{
    const DevMesh &m = C.m;
    if (!m.wall_stats || m.n_wall == 0) return;
    k_wall_stats<T><<<cdiv(m.n_wall, 128), 128, 0, s>>>((const T *)m.g[m.gcur], m.Np, m.n_wall, m.wall_ns, m.wall_acc,
                                                        1.0 / (0.5 * C.u0 * C.u0));
}

template <typename T, typename S> void launch_mass(const DevCtx &C, double *row_sum, double *out, cudaStream_t s)
{
    const DevLevel &l = C.lv[0];
    if (l.parity == 0)
        k_mass_rows<T, S, 0><<<l.ny, kMassThreads, 0, s>>>((const S *)l.f, l.nx, l.pitch, l.stride, l.hx0, l.hx1,
                                                           row_sum, C.shift);
    else
        k_mass_rows<T, S, 1><<<l.ny, kMassThreads, 0, s>>>((const S *)l.f, l.nx, l.pitch, l.stride, l.hx0, l.hx1,
                                                           row_sum, C.shift);
    k_mass_total<<<1, kMassThreads, 0, s>>>(row_sum, l.ny, out);
}

template <typename T, typename S>
void launch_fields(const DevCtx &C, int grid, double *rho, double *ux, double *uy, double *pop, cudaStream_t s)
{
    if (grid < 0) {
        const DevMesh &m = C.m;
        k_fields_mesh<T><<<cdiv(m.n, 128), 128, 0, s>>>((const T *)m.g[m.gcur], m.Np, m.inv, m.n, rho, ux, uy, pop);
        return;
    }
    const DevLevel &l = C.lv[grid];
    dim3 g(cdiv(l.nx, 128), l.ny);
    if (l.parity == 0)
        k_fields_level<T, S, 0><<<g, 128, 0, s>>>((const S *)l.f, l.nx, l.ny, l.pitch, l.stride, l.hx0, l.hx1, rho, ux,
                                                  uy, pop, C.shift);
    else
        k_fields_level<T, S, 1><<<g, 128, 0, s>>>((const S *)l.f, l.nx, l.ny, l.pitch, l.stride, l.hx0, l.hx1, rho, ux,
                                                  uy, pop, C.shift);
}

#define HLBM_INSTANTIATE(T, S)                                                                                   \
    template void configure_fv<T, S>(const FvTiles &);                                                           \
    template void configure_fv_prefetch<T, S>(FvTiles &);                                                        \
    template void launch_init_level<T, S>(const DevCtx &, int, unsigned long long, double, cudaStream_t);        \
    template void launch_collide<T, S>(const DevCtx &, int, cudaStream_t);                                       \
    template void launch_outer_bc<T, S>(const DevCtx &, cudaStream_t);                                           \
    template void launch_snapshot<T, S>(const DevCtx &, int, bool, cudaStream_t);                                \
    template void launch_prolong<T, S>(const DevCtx &, int, double, cudaStream_t);                               \
    template void launch_restrict<T, S>(const DevCtx &, int, cudaStream_t);                                      \
    template void launch_ring_interp<T, S>(const DevCtx &, bool, cudaStream_t);                                  \
    template void launch_hole_interp<T, S>(const DevCtx &, cudaStream_t);                                        \
    template void launch_fv<T, S>(const DevCtx &, int, cudaStream_t);                                            \
    template void launch_fv_filter<T, S>(const DevCtx &, cudaStream_t);                                         \
    template int fv_autotune<T, S>(DevCtx &, cudaStream_t, double *);                                            \
    template void launch_forces<T, S>(const DevCtx &, cudaStream_t);                                             \
    template void launch_mass<T, S>(const DevCtx &, double *, double *, cudaStream_t);                           \
    template void launch_wall_stats<T, S>(const DevCtx &, cudaStream_t);                                         \
    template void launch_fields<T, S>(const DevCtx &, int, double *, double *, double *, double *, cudaStream_t);
HLBM_INSTANTIATE(float, float)
HLBM_INSTANTIATE(double, double)
HLBM_INSTANTIATE(float, __half)

}  // namespace hlbm
