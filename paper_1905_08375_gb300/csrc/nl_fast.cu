// nl_fast.cu -- the fast algorithm of Sec. 3 for polynomial kernels
//   P(x, y) = sigma C(x) delta(x)^{-(d+2)} p^{2K}(|y - x| / delta(x)).
//
// Step 2 (bottom-up partial sums): a pyramid of panel moments in FP64.  At
// the leaves (one node per leaf cell, at its centre) the moments are v_k and
// zeros; a parent's moments are its children's re-expanded about the parent
// centre (binomial shift, exact algebra), in the coordinates
// t = (x - c_Q) / (w_Q / 2) so that every moment is O(|v|).
//
// Step 1 + Step 3: the decomposition of Algorithm 1 is not stored.  A panel Q
// of level l is in the decomposition of node x iff its parent is not fully
// inside the ball and either Q is fully inside (all corners strictly inside,
// the containment test of Algorithm 1) or Q is a leaf that meets the open
// ball (Algorithm 2).  For a fixed panel row both conditions select one
// contiguous run of panels whose end points follow from an integer square
// root, so each node enumerates its decomposition level by level, row by row,
// as at most two runs per row, and sums Eq. (3.5) over those panels.
//
// Geometry is exact integer arithmetic in half-units of h: node i sits at
// X = 2 i + 1, panel k of level l spans [k S, (k + 1) S] with S = 2^{L-l+1},
// and the ball test is (squared distance) <= thr4_i, thr4_i the largest
// integer below 4 R2_i.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "nl_internal.cuh"

namespace {

__device__ __forceinline__ int floor_div(int a, int b)   // b > 0
{
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}
__device__ __forceinline__ int ceil_div(int a, int b) { return -floor_div(-a, b); }

// largest r >= 0 with r*r <= x (x >= 0)
__device__ __forceinline__ int isqrt_floor(int x)
{
    int r = (int)sqrtf((float)x);
    while (r > 0 && (long long)r * r > x) --r;
    while ((long long)(r + 1) * (r + 1) <= x) ++r;
    return r;
}

// farthest / nearest squared distance (half-units) from X to panel [kS, (k+1)S]
__device__ __forceinline__ int far2(int k, int S, int X)
{
    const int a = abs(k * S - X), b = abs((k + 1) * S - X);
    const int m = a > b ? a : b;
    return m * m;
}
__device__ __forceinline__ int near2(int k, int S, int X)
{
    int g = 0;
    if (k * S > X) g = k * S - X;
    else if ((k + 1) * S < X) g = X - (k + 1) * S;
    return g * g;
}

struct FastArgs {
    int d, n, L, K, M;
    int64_t N;
    const int *thr4;
    const double *fastF, *selfS, *ir4;
    const double *pyr;           // levels 0..L-1, [panel][M]
    const double *leaf;          // level L, v_k
    int64_t lvl_off[NL_MAX_LEVELS + 2];
    double hd;
    double poly[8];
};

// moment index of (a0, a1) in the compact order (a1 outer, a0 inner, a0 + a1 <= 2K)
template <int K>
__device__ __host__ __forceinline__ int midx2(int a0, int a1)
{
    return a1 * (2 * K + 1) - (a1 * (a1 - 1)) / 2 + a0;
}

// moment index of (a0, a1, a2) in the compact order (a2 outer, a1, a0 inner, sum <= 2K)
template <int K>
__device__ __host__ __forceinline__ constexpr int midx3(int a0, int a1, int a2)
{
    int idx = 0;
    for (int c = 0; c < a2; ++c) idx += (2 * K - c + 1) * (2 * K - c + 2) / 2;
    for (int b = 0; b < a1; ++b) idx += 2 * K - a2 - b + 1;
    return idx + a0;
}

// sum over x_k in panel of p(|x_k - x_i|^2 / delta_i^2) v_k from the panel moments:
// |x_k - x_i|^2 / delta^2 = |B + H t|^2 / (4 R2), B = centre - X, H = half-width
template <int D, int K>
__device__ __forceinline__ double panel_poly(const double *mu, const double *pc, int Bx, int By,
                                             int Bz, int H, double ir4)
{
    if constexpr (K == 0) {
        return pc[0] * mu[0];
    } else if constexpr (D == 3) {
        // q(t) = p(|B + H t|^2 ir4) as a polynomial in (t0, t1, t2) of degree 2K, by Horner's
        // rule in s = c000 + sum_a c_a t_a + H2 sum_a t_a^2, kept in the compact moment order
        // (runtime loops: up to 84 coefficients, so the arrays live in local memory)
        constexpr int M = (2 * K + 1) * (2 * K + 2) * (2 * K + 3) / 6;
        const double H2 = (double)H * H * ir4;
        const double c000 = ((double)Bx * Bx + (double)By * By + (double)Bz * Bz) * ir4;
        const double c1[3] = { 2.0 * Bx * H * ir4, 2.0 * By * H * ir4, 2.0 * Bz * H * ir4 };
        double q[M], nq[M];
#pragma unroll 1
        for (int e = 0; e < M; ++e) q[e] = 0.0;
        q[0] = pc[K];
#pragma unroll 1
        for (int m = K - 1; m >= 0; --m) {
            int e = 0;
#pragma unroll 1
            for (int c = 0; c <= 2 * K; ++c)
#pragma unroll 1
                for (int b = 0; b <= 2 * K - c; ++b)
#pragma unroll 1
                    for (int a0 = 0; a0 <= 2 * K - b - c; ++a0, ++e) {
                        double v = c000 * q[e];
                        if (a0 >= 1) v += c1[0] * q[e - 1];
                        if (b >= 1) v += c1[1] * q[midx3<K>(a0, b - 1, c)];
                        if (c >= 1) v += c1[2] * q[midx3<K>(a0, b, c - 1)];
                        if (a0 >= 2) v += H2 * q[e - 2];
                        if (b >= 2) v += H2 * q[midx3<K>(a0, b - 2, c)];
                        if (c >= 2) v += H2 * q[midx3<K>(a0, b, c - 2)];
                        nq[e] = v;
                    }
            nq[0] += pc[m];
#pragma unroll 1
            for (int f = 0; f < M; ++f) q[f] = nq[f];
        }
        double v = 0.0;
#pragma unroll 1
        for (int e = 0; e < M; ++e) v += q[e] * mu[e];
        return v;
    } else if constexpr (D == 1) {
        constexpr int E = 2 * K + 1;
        const double c0 = (double)Bx * Bx * ir4, c1 = 2.0 * Bx * H * ir4, c2 = (double)H * H * ir4;
        double q[E];
#pragma unroll
        for (int e = 0; e < E; ++e) q[e] = 0.0;
        q[0] = pc[K];
#pragma unroll
        for (int m = K - 1; m >= 0; --m) {
            // q <- q * (c0 + c1 t + c2 t^2) + p_m; degree grows by 2 each step
            double nq[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                double s = c0 * q[e];
                if (e >= 1) s += c1 * q[e - 1];
                if (e >= 2) s += c2 * q[e - 2];
                nq[e] = s;
            }
            nq[0] += pc[m];
#pragma unroll
            for (int e = 0; e < E; ++e) q[e] = nq[e];
        }
        double v = 0.0;
#pragma unroll
        for (int e = 0; e < E; ++e) v += q[e] * mu[e];
        return v;
    } else {
        constexpr int E = 2 * K + 1;
        const double H2 = (double)H * H * ir4;
        const double c00 = ((double)Bx * Bx + (double)By * By) * ir4;
        const double c10 = 2.0 * Bx * H * ir4, c01 = 2.0 * By * H * ir4;
        double q[E][E];
#pragma unroll
        for (int a = 0; a < E; ++a)
#pragma unroll
            for (int b = 0; b < E; ++b) q[a][b] = 0.0;
        q[0][0] = pc[K];
#pragma unroll
        for (int m = K - 1; m >= 0; --m) {
            double nq[E][E];
#pragma unroll
            for (int a = 0; a < E; ++a)
#pragma unroll
                for (int b = 0; b < E; ++b) {
                    double s = 0.0;
                    if (a + b <= 2 * K) {
                        s = c00 * q[a][b];
                        if (a >= 1) s += c10 * q[a - 1][b];
                        if (b >= 1) s += c01 * q[a][b - 1];
                        if (a >= 2) s += H2 * q[a - 2][b];
                        if (b >= 2) s += H2 * q[a][b - 2];
                    }
                    nq[a][b] = s;
                }
            nq[0][0] += pc[m];
#pragma unroll
            for (int a = 0; a < E; ++a)
#pragma unroll
                for (int b = 0; b < E; ++b) q[a][b] = nq[a][b];
        }
        double v = 0.0;
#pragma unroll
        for (int b = 0; b < E; ++b)
#pragma unroll
            for (int a = 0; a + b < E; ++a) v += q[a][b] * mu[midx2<K>(a, b)];
        return v;
    }
}

// Parent-full x-range (child units) of parent row (pky, pkz) at level l-1, or empty.
__device__ __forceinline__ void parent_full(int D, int l, int S, int np, int X, int Y, int Z,
                                            int ky, int kz, int T4, int &lo, int &hi)
{
    lo = 1; hi = 0;
    if (l == 0) return;
    const int S2 = 2 * S, npp = np >> 1;
    int e = 0;
    if (D > 1) e += far2(ky >> 1, S2, Y);
    if (D > 2) e += far2(kz >> 1, S2, Z);
    if (e > T4) return;
    const int r = isqrt_floor(T4 - e);
    const int a = max(0, ceil_div(X - r, S2));
    const int b = min(npp - 1, floor_div(X + r, S2) - 1);
    if (a > b) return;
    lo = 2 * a;
    hi = 2 * b + 1;
}

template <int D, int K>
__device__ __forceinline__ double sum_run(const FastArgs &a, int l, int np, int S, int ka, int kb,
                                          int ky, int kz, int X, int Y, int Z, int ix, int iy,
                                          int iz, double ir4)
{
    double s = 0.0;
    if (ka > kb) return s;
    const int64_t rowbase = (int64_t)np * (ky + (int64_t)np * kz);
    if (l == a.L) {
        const double *leaf = a.leaf + rowbase;
        if constexpr (K == 0) {
            for (int k = ka; k <= kb; ++k) s += leaf[k];
        } else {
            const int oy = ky - iy, oz = kz - iz;
            for (int k = ka; k <= kb; ++k) {
                const int ox = k - ix;
                const double t = (double)(ox * ox + oy * oy + oz * oz) * (4.0 * ir4);
                double w = a.poly[K];
#pragma unroll
                for (int m = K - 1; m >= 0; --m) w = w * t + a.poly[m];
                s += w * leaf[k];
            }
        }
    } else {
        const double *lev = a.pyr + a.lvl_off[l] + rowbase * a.M;
        if constexpr (K == 0) {
            for (int k = ka; k <= kb; ++k) s += lev[k];
        } else {
            const int H = S / 2;
            const int By = (D > 1) ? ky * S + H - Y : 0;
            const int Bz = (D > 2) ? kz * S + H - Z : 0;
            for (int k = ka; k <= kb; ++k) {
                const int Bx = k * S + H - X;
                s += panel_poly<D, K>(lev + (int64_t)k * a.M, a.poly, Bx, By, Bz, H, ir4);
            }
        }
    }
    return s;
}

template <int D, int K, typename T>
__global__ void __launch_bounds__(256) k_fast_gather(FastArgs a, const T *__restrict__ u,
                                                     T *__restrict__ Lu)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int n = a.n;
    const int ix = (int)(i % n);
    const int iy = D > 1 ? (int)((i / n) % n) : 0;
    const int iz = D > 2 ? (int)(i / ((int64_t)n * n)) : 0;
    const int X = 2 * ix + 1, Y = 2 * iy + 1, Z = 2 * iz + 1;
    const int T4 = a.thr4[i];
    const double ir4 = (K > 0) ? a.ir4[i] : 0.0;
    const int r0 = isqrt_floor(T4);
    double G = 0.0;
    for (int l = 0; l <= a.L; ++l) {
        const int np = 1 << l;
        const int S = 2 << (a.L - l);
        const bool leaf = (l == a.L);
        // rows (and slabs) that can hold included panels at this level
        int ylo = 0, yhi = 0, zlo = 0, zhi = 0;
        if (D > 1) {
            ylo = max(0, leaf ? ceil_div(Y - r0, S) - 1 : ceil_div(Y - r0, S));
            yhi = min(np - 1, leaf ? floor_div(Y + r0, S) : floor_div(Y + r0, S) - 1);
        }
        if (D > 2) {
            zlo = max(0, leaf ? ceil_div(Z - r0, S) - 1 : ceil_div(Z - r0, S));
            zhi = min(np - 1, leaf ? floor_div(Z + r0, S) : floor_div(Z + r0, S) - 1);
        }
        for (int kz = zlo; kz <= zhi; ++kz) {
            const int ez_far = D > 2 ? far2(kz, S, Z) : 0;
            const int ez_near = D > 2 ? near2(kz, S, Z) : 0;
            for (int ky = ylo; ky <= yhi; ++ky) {
                const int e_far = ez_far + (D > 1 ? far2(ky, S, Y) : 0);
                const int e_near = ez_near + (D > 1 ? near2(ky, S, Y) : 0);
                int ka, kb;
                if (leaf) {
                    if (e_near > T4) continue;
                    const int r = isqrt_floor(T4 - e_near);
                    ka = max(0, ceil_div(X - r, S) - 1);
                    kb = min(np - 1, floor_div(X + r, S));
                } else {
                    if (e_far > T4) continue;
                    const int r = isqrt_floor(T4 - e_far);
                    ka = max(0, ceil_div(X - r, S));
                    kb = min(np - 1, floor_div(X + r, S) - 1);
                }
                if (ka > kb) continue;
                int pa, pb;
                parent_full(D, l, S, np, X, Y, Z, ky, kz, T4, pa, pb);
                if (pa > pb) {
                    G += sum_run<D, K>(a, l, np, S, ka, kb, ky, kz, X, Y, Z, ix, iy, iz, ir4);
                } else {
                    G += sum_run<D, K>(a, l, np, S, ka, min(kb, pa - 1), ky, kz, X, Y, Z, ix, iy, iz, ir4);
                    G += sum_run<D, K>(a, l, np, S, max(ka, pb + 1), kb, ky, kz, X, Y, Z, ix, iy, iz, ir4);
                }
            }
        }
    }
    const double ui = (double)u[i];
    Lu[i] = (T)(a.fastF[i] * (a.hd * G - ui * a.selfS[i]));
}

// ---------------------------------------------------------------------------
// Step 2: the moment pyramid
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_pyr_leaf(int64_t N, const T *__restrict__ u, const double *__restrict__ b,
                           double *leaf)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) leaf[i] = (double)u[i] * b[i];
}

// one thread per parent panel of level l; children at level l+1
__global__ void k_pyr_level(int d, int l, int L, int M, const double *__restrict__ child,
                            double *__restrict__ parent, const double *__restrict__ shift)
{
    const int np = 1 << l;
    int64_t P = np;
    if (d > 1) P *= np;
    if (d > 2) P *= np;
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= P) return;
    const int kx = (int)(f % np);
    const int ky = d > 1 ? (int)((f / np) % np) : 0;
    const int kz = d > 2 ? (int)(f / ((int64_t)np * np)) : 0;
    const int nc = 2 * np;
    const bool child_leaf = (l + 1 == L);
    const int cm = child_leaf ? 1 : M;       // leaves carry v only
    for (int al = 0; al < M; ++al) {
        double acc = 0.0;
        for (int s = 0; s < (1 << d); ++s) {
            const int cx = 2 * kx + (s & 1);
            const int cy = d > 1 ? 2 * ky + ((s >> 1) & 1) : 0;
            const int cz = d > 2 ? 2 * kz + ((s >> 2) & 1) : 0;
            const int64_t fc = cx + (int64_t)nc * (cy + (int64_t)nc * cz);
            const double *mu = child + fc * cm;
            const double *T = shift + ((int64_t)s * M + al) * M;
            for (int be = 0; be < cm; ++be) acc += T[be] * mu[be];
        }
        parent[f * M + al] = acc;
    }
}

// self term S_i of Eq. (3.3) (plan time) and per-node factors
__global__ void k_fast_node(int d, int n, int K, int coef, int self_mode, int64_t N, double sigma,
                            double sphere, const double *__restrict__ delta,
                            const double *__restrict__ acoef, const int *__restrict__ thr4,
                            const double *__restrict__ pc, double *fastF, double *selfS,
                            double *ir4)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double di = delta[i];
    const double rho = di * n;
    const double R2 = rho * rho;
    const double ai = acoef ? acoef[i] : 1.0;
    const double Ai = (coef == NL_COEF_NONE) ? 1.0 : ai;
    fastF[i] = sigma * Ai * pow(di, -(d + 2.0));
    ir4[i] = 1.0 / (4.0 * R2);
    if (self_mode == NL_SELF_PAPER) {
        double s = 0.0;
        for (int m = 0; m <= K; ++m) s += pc[m] / (2.0 * m + d);
        selfS[i] = sphere * pow(di, (double)d) * s;
        return;
    }
    const int ix = (int)(i % n);
    const int iy = d > 1 ? (int)((i / n) % n) : 0;
    const int iz = d > 2 ? (int)(i / ((int64_t)n * n)) : 0;
    const int T4 = thr4[i];
    const int B = (int)ceil(rho) + 1;
    const int bz = d > 2 ? B : 0, by = d > 1 ? B : 0;
    double acc = 0.0;
    for (int oz = -bz; oz <= bz; ++oz)
        for (int oy = -by; oy <= by; ++oy)
            for (int ox = -B; ox <= B; ++ox) {
                // gap from the node (cell centre) to cell i + o, half-units: 2|o| - 1
                const int gx = ox ? 2 * abs(ox) - 1 : 0;
                const int gy = oy ? 2 * abs(oy) - 1 : 0;
                const int gz = oz ? 2 * abs(oz) - 1 : 0;
                if (gx * gx + gy * gy + gz * gz > T4) continue;
                double b = 1.0;
                if (coef == NL_COEF_XY) {
                    const int jx = ix + ox, jy = iy + oy, jz = iz + oz;
                    bool in = jx >= 0 && jx < n;
                    if (d > 1) in = in && jy >= 0 && jy < n;
                    if (d > 2) in = in && jz >= 0 && jz < n;
                    b = in ? acoef[jx + (int64_t)n * (jy + (int64_t)n * jz)] : ai;
                }
                const double t = (double)(ox * ox + oy * oy + oz * oz) / R2;
                double w = pc[K];
                for (int m = K - 1; m >= 0; --m) w = w * t + pc[m];
                acc += w * b;
            }
    selfS[i] = pow(1.0 / n, (double)d) * acc;
}

// ---------------------------------------------------------------------------
// p^0 = 1 with FP32 data: Step 2 partial sums in 64-bit fixed point.  One reduction finds
// m = max |v|; with S = 62 - ceil(log2(N m)) every leaf value is rounded once to an integer
// multiple of 2^-S and every partial sum of any set of leaves is then exact (|sum| < 2^62).
// Step 3 adds the integer panel sums of the decomposition exactly, panel by panel.
// ---------------------------------------------------------------------------
// floor(sqrt(x)) for 0 <= x < 2^30: one approximate reciprocal square root (relative error
// well below 2^-20, so the estimate is within 1 of the answer), then exact integer corrections
__device__ __forceinline__ int isqrt_fast(int x)
{
    const float f = (float)max(x, 1);
    int h = __float2int_rz(f * rsqrtf(f));
    h -= (h * h > x);
    h += ((h + 1) * (h + 1) <= x);
    return h;
}


// scale exponent S with N * max|v| * 2^S < 2^62, from the FP32 bound
__device__ __forceinline__ int fixed_shift_f32(int64_t N, const unsigned int *mx)
{
    const float m = __uint_as_float(*mx);
    if (!(m > 0.f)) return 62;
    int e1, e2;
    frexpf(m, &e1);                     // m < 2^e1
    frexpf((float)N, &e2);              // N < 2^e2
    return 62 - e1 - e2;
}

// The self term joins the exact integer sum: with selfQ = selfS / h^d and Fh = fastF h^d,
//   out = fastF (h^d G 2^-S - u selfS) = Fh 2^-S (G - u selfQ 2^S),
// T = round(u selfQ 2^S) (one more rounding at the scale of the leaf values), D = G - T exact,
// then D is scaled in FP32.  Where |u selfQ 2^S| could leave 64 bits the FP64 form is used.
__device__ __forceinline__ float fixed_epilogue(long long G, float u, double selfQ, float Fh,
                                                double fastF, double selfS, double hd, int sh)
{
    const double s2 = __longlong_as_double((long long)(sh + 1023) << 52);     // 2^sh
    const double t = (double)u * selfQ * s2;
    if (fabs(t) < 0x1p62) {
        const long long D = G - __double2ll_rn(t);
        return ldexpf(Fh * (float)D, -sh);
    }
    return (float)(fastF * (hd * ldexp((double)G, -sh) - (double)u * selfS));
}

__global__ void k_fixed_consts(int64_t N, double hd, const double *__restrict__ fastF,
                               const double *__restrict__ selfS, double *__restrict__ selfQ,
                               float *__restrict__ Fh)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    selfQ[i] = selfS[i] / hd;
    Fh[i] = (float)(fastF[i] * hd);
}




struct FastI64Args {
    int n, L;
    int64_t N;
    const int *thr4;
    const double *fastF, *selfS, *selfQ;
    const float *Fh;
    const long long *pyr;                  // levels 0..L (leaf level last), panel-major
    int64_t lvl_off[NL_MAX_LEVELS + 2];
    double hd;
    const unsigned int *mx;
};

__device__ __forceinline__ int sq(int v) { return v * v; }

template <int D, typename T>
__global__ void __launch_bounds__(256) k_fast_gather_i64(FastI64Args a, const T *__restrict__ u,
                                                         T *__restrict__ Lu)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int n = a.n, L = a.L;
    const int ix = (int)(i % n);
    const int iy = D > 1 ? (int)((i / n) % n) : 0;
    const int iz = D > 2 ? (int)(i / ((int64_t)n * n)) : 0;
    const int X = 2 * ix + 1, Y = 2 * iy + 1, Z = 2 * iz + 1;
    const int T4 = a.thr4[i];
    const int r0 = isqrt_fast(T4);
    long long G = 0;
    for (int l = 0; l <= L; ++l) {
        const int np = 1 << l;
        const int sh = L - l + 1;          // panel size 2^sh half-units
        const bool leaf = (l == L);
        const long long *lev = a.pyr + a.lvl_off[l];
        // distances from the node to panel k's interval along one axis (half-units):
        //   far(k) = max(|k S - X|, |(k+1) S - X|), near(k) = gap or 0
        int ylo = 0, yhi = 0, zlo = 0, zhi = 0;
        if (D > 1) {
            ylo = max(0, leaf ? ((Y - r0) >> sh) : -((r0 - Y) >> sh));
            yhi = min(np - 1, ((Y + r0) >> sh) - (leaf ? 0 : 1));
            if (leaf) ylo = max(0, -((r0 - Y) >> sh) - 1);
        }
        if (D > 2) {
            zlo = leaf ? max(0, -((r0 - Z) >> sh) - 1) : max(0, -((r0 - Z) >> sh));
            zhi = min(np - 1, ((Z + r0) >> sh) - (leaf ? 0 : 1));
        }
        for (int kz = zlo; kz <= zhi; ++kz) {
            const int z0 = (kz << sh) - Z, z1 = z0 + (1 << sh);
            const int ez = D > 2 ? (leaf ? (z0 > 0 ? sq(z0) : (z1 < 0 ? sq(z1) : 0))
                                         : max(sq(z0), sq(z1))) : 0;
            const int pz0 = ((kz >> 1) << (sh + 1)) - Z, pz1 = pz0 + (2 << sh);
            const int epz = D > 2 ? max(sq(pz0), sq(pz1)) : 0;
            for (int ky = ylo; ky <= yhi; ++ky) {
                const int y0 = (ky << sh) - Y, y1 = y0 + (1 << sh);
                int e = ez;
                if (D > 1) e += leaf ? (y0 > 0 ? sq(y0) : (y1 < 0 ? sq(y1) : 0))
                                     : max(sq(y0), sq(y1));
                if (e > T4) continue;
                const int r = isqrt_fast(T4 - e);
                int ka, kb;
                if (leaf) {
                    ka = max(0, -((r - X) >> sh) - 1);
                    kb = min(np - 1, (X + r) >> sh);
                } else {
                    ka = max(0, -((r - X) >> sh));
                    kb = min(np - 1, ((X + r) >> sh) - 1);
                }
                if (ka > kb) continue;
                int pa = 1, pb = 0;               // parent row's fully-inside panels
                if (l > 0) {
                    const int py0 = ((ky >> 1) << (sh + 1)) - Y, py1 = py0 + (2 << sh);
                    const int ep = epz + (D > 1 ? max(sq(py0), sq(py1)) : 0);
                    if (ep <= T4) {
                        const int rp = isqrt_fast(T4 - ep);
                        const int qa = max(0, -((rp - X) >> (sh + 1)));
                        const int qb = min((np >> 1) - 1, ((X + rp) >> (sh + 1)) - 1);
                        if (qa <= qb) { pa = 2 * qa; pb = 2 * qb + 1; }
                    }
                }
                const long long *row = lev + (int64_t)np * (ky + (int64_t)np * kz);
                const int e1 = min(kb, pa - 1);
                for (int k = ka; k <= e1; ++k) G += row[k];
                for (int k = max(ka, pb + 1); k <= kb; ++k) G += row[k];
            }
        }
    }
    const int sh = fixed_shift_f32(a.N, a.mx);
    Lu[i] = (T)fixed_epilogue(G, (float)u[i], a.selfQ[i], a.Fh[i], a.fastF[i], a.selfS[i], a.hd, sh);
}

// ---------------------------------------------------------------------------
// Row-prefix form of the integer partial sums: at every level, P[k] holds the sum of the
// panels 0..k of its panel row, so the panels ka..kb of a run add up to P[kb] - P[ka-1],
// exactly the same integer as adding them one by one.  The leaf rows are scanned; a
// parent's prefix is the sum of its child rows' prefixes at the odd positions.
// k_step2_rowprefix (below) builds all the levels in one launch.
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// Step 2 of the row-prefix form in two launches.  k_absmax_parts writes one bound of |u b| per
// block and zeroes the coarse levels 0 .. lf-1.  k_step2_rowprefix, one block per band (a
// band is the set of leaf rows of one panel row of level lf), then (1) reduces the bounds to
// the scale exponent, quantises and scans the band's leaf rows (a warp per row), (2) builds
// the levels L-1 .. lf of the band, and (3) adds the band's part of every coarser prefix,
// P_l[row][k] += P_lf[band][(k + 1) 2^(lf-l) - 1], with integer atomics.  Every value is the
// prefix of the panel sums of its row (integer sums are exact and do not depend on the
// order in which the atomics land).
// ---------------------------------------------------------------------------
// One bound of |u b| per block, from max |u| and the plan-time bound bmax = max |b| (only u
// is read): |fl32(u b)| <= max|u| bmax (1 + 2^-24), below fl32(max|u| bmax) (1 + 2^-20).
__global__ void __launch_bounds__(256) k_absmax_parts(int64_t N, const float *__restrict__ u,
                                                      float bmax,
                                                      float *__restrict__ part,
                                                      long long *__restrict__ zero,
                                                      int64_t nzero)
{
    __shared__ float s_w[8];
    float m = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < nzero; i += stride) zero[i] = 0;
    int64_t done = 0;
    if ((reinterpret_cast<uintptr_t>(u) & 15) == 0) {
        // 16-byte loads, eight in flight per thread
        const float4 *__restrict__ u4 = reinterpret_cast<const float4 *>(u);
        const int64_t N4 = N >> 2;
        for (int64_t i = t0; i < N4; i += 8 * stride) {
            float4 x[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int64_t j = i + q * stride;
                x[q] = j < N4 ? u4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
                m = fmaxf(fmaxf(m, fmaxf(fabsf(x[q].x), fabsf(x[q].y))),
                          fmaxf(fabsf(x[q].z), fabsf(x[q].w)));
        }
        done = N4 << 2;
    }
    for (int64_t i = done + t0; i < N; i += stride) m = fmaxf(m, fabsf(u[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmaxf(m, s_w[w]);
        part[blockIdx.x] = (m * bmax) * (1.f + 0x1p-20f);
    }
}

// max |b| over the nodes (plan time), as the bits of a non-negative float
__global__ void k_max_abs_bits(int64_t N, const float *__restrict__ b, unsigned int *out)
{
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(b[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

constexpr int LEAF_MULTI = 8;
constexpr int LEAF_MULTI_MAX = LEAF_MULTI;

struct Step2Args {
    int d, n, L, c, lf;              // band: 2^c leaf rows per axis = one panel row of level lf
    int leaf_only;                   // 1: the leaf rows only (leaf-row gather)
    int wpr;                         // warps per leaf row (leaf rows only; n / 256 when > 1)
    int vec;                         // panel sums: u, b and the leaf level 16-byte aligned,
                                     // n a multiple of 4 (16-byte loads and stores)
    int lane_e;                      // leaf rows only, n = 32 lane_e (4 or 8) with 16-byte
                                     // aligned u and b: lane l holds nodes lane_e l .. + lane_e-1
    int64_t N;
    const float *u, *b;
    const float *part;
    int nparts;
    unsigned int *mx;
    long long *pyr;
    long long *leaf;                 // the leaf level (pyr + lvl_off[L], or a separate buffer)
    int64_t lvl_off[NL_MAX_LEVELS + 2];
};

__device__ __forceinline__ long long warp_incl_scan_ll(long long v, int lane)
{
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// parent prefix at (kx, ky, kz) of level l from level l + 1 (child rows at odd positions)
__device__ __forceinline__ long long level_prefix_at(int d, int l, const long long *child,
                                                     int kx, int ky, int kz)
{
    const int nc = 2 << l;
    long long s = 0;
    for (int c = 0; c < (1 << (d - 1)); ++c) {
        const int cy = d > 1 ? 2 * ky + (c & 1) : 0;
        const int cz = d > 2 ? 2 * kz + ((c >> 1) & 1) : 0;
        s += __ldcg(child + (2 * kx + 1) + (int64_t)nc * (cy + (int64_t)nc * cz));
    }
    return s;
}

constexpr int STEP2_THREADS = 512;

__global__ void __launch_bounds__(1024) k_step2_rowprefix(Step2Args a)
{
    __shared__ float s_w[32];                    // one bound per warp (up to 1024 threads)
    const int nt = blockDim.x;                   // STEP2_THREADS, or 128 for the leaf rows only
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = nt / 32;
    // scale exponent from the per-block bounds (same arithmetic as fixed_shift_f32)
    float m = 0.f;
    for (int k = tid; k < a.nparts; k += nt) m = fmaxf(m, a.part[k]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) s_w[warp] = m;
    __syncthreads();
    m = 0.f;
    for (int w = 0; w < nw; ++w) m = fmaxf(m, s_w[w]);
    if (blockIdx.x == 0 && tid == 0) *a.mx = __float_as_uint(m);
    int sh = 62;
    if (m > 0.f) {
        int e1, e2;
        frexpf(m, &e1);
        frexpf((float)a.N, &e2);
        sh = 62 - e1 - e2;
    }
    const int n = a.n, d = a.d, L = a.L, lf = a.lf;
    const int S = 1 << a.c;                    // band side in leaf rows (per axis)
    const int bands_y = d > 1 ? n / S : 1;
    const int by = d > 1 ? (int)(blockIdx.x % bands_y) : 0;
    const int bz = d > 2 ? (int)(blockIdx.x / bands_y) : 0;
    const int rows_y = d > 1 ? S : 1, rows_z = d > 2 ? S : 1;
    long long *leaf = a.leaf;
    // (1) quantise and scan the band's leaf rows.  a.wpr > 1 (the leaf rows alone, n >= 512):
    // a row is split among wpr warps of 256 nodes (eight 32-node pages each, kept in
    // registers); each warp's total goes to shared memory and the later segments add the
    // earlier ones' totals before storing.  Otherwise one warp per row, the 32 loads of a
    // 1024-node page issued first, the page scanned 32 nodes at a time.
    if (a.lane_e) {
        // n = 32 E: each lane loads its E consecutive nodes with 16-byte loads, scans them in
        // registers, one warp scan of the lane totals gives the offsets, and the row is stored
        // through shared memory so that the 8-byte stores are coalesced
        __shared__ long long s_row[4 * 256];      // at most four warps of n <= 256
        const int E = a.lane_e;
        long long *srow = s_row + warp * n;
        for (int r = warp; r < rows_y * rows_z; r += nw) {
            const int iy = by * rows_y + r % rows_y, iz = bz * rows_z + r / rows_y;
            const int64_t row = (int64_t)n * (iy + (int64_t)n * iz);
            const float4 *__restrict__ u4 = reinterpret_cast<const float4 *>(a.u + row) + lane * (E / 4);
            const float4 *__restrict__ b4 = reinterpret_cast<const float4 *>(a.b + row) + lane * (E / 4);
            float v[8];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (4 * k < E) {
                    const float4 x = u4[k], y = b4[k];
                    v[4 * k] = x.x * y.x; v[4 * k + 1] = x.y * y.y;
                    v[4 * k + 2] = x.z * y.z; v[4 * k + 3] = x.w * y.w;
                }
            }
            long long q[8], t = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (k < E) {
                    t += __float2ll_rn(ldexpf(v[k], sh));
                    q[k] = t;
                }
            }
            long long off = warp_incl_scan_ll(t, lane) - t;        // exclusive lane offset
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (k < E) srow[E * lane + k] = q[k] + off;
            __syncwarp();
            for (int x = lane; x < n; x += 32) leaf[row + x] = srow[x];
            __syncwarp();
        }
    } else if (a.wpr > 1) {
        __shared__ long long s_tot[32];
        const int W = a.wpr, part = warp % W, r = warp / W;     // one row per W warps
        const int iy = by * rows_y + r % rows_y, iz = bz * rows_z + r / rows_y;
        const int64_t row = (int64_t)n * (iy + (int64_t)n * iz) + 256 * part;
        const float *__restrict__ ur = a.u + row;
        const float *__restrict__ br = a.b + row;
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = ur[32 * k + lane] * br[32 * k + lane];
        long long q[8], carry = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            long long t = __float2ll_rn(ldexpf(v[k], sh));
            for (int o = 1; o < 32; o <<= 1) {
                const long long w = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += w;
            }
            q[k] = t + carry;
            carry = __shfl_sync(0xffffffffu, q[k], 31);
        }
        if (lane == 0) s_tot[warp] = carry;
        __syncthreads();
        long long off = 0;
        for (int w = warp - part; w < warp; ++w) off += s_tot[w];
#pragma unroll
        for (int k = 0; k < 8; ++k) leaf[row + 32 * k + lane] = q[k] + off;
    } else
    for (int r = warp; r < rows_y * rows_z; r += nw) {
        const int iy = by * rows_y + r % rows_y, iz = bz * rows_z + r / rows_y;
        const int64_t row = (int64_t)n * (iy + (int64_t)n * iz);
        const float *__restrict__ ur = a.u + row;
        const float *__restrict__ br = a.b + row;
        long long carry = 0;
        for (int p0 = 0; p0 < n; p0 += 1024) {
            float v[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int x = p0 + 32 * k + lane;
                v[k] = x < n ? ur[x] * br[x] : 0.f;
            }
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                if (p0 + 32 * k >= n) break;
                const int x = p0 + 32 * k + lane;
                long long q = x < n ? __float2ll_rn(ldexpf(v[k], sh)) : 0LL;
                q = warp_incl_scan_ll(q, lane) + carry;
                if (x < n) leaf[row + x] = q;
                carry = __shfl_sync(0xffffffffu, q, 31);
            }
        }
    }
    if (a.leaf_only) return;
    __syncthreads();
    // (2) levels L-1 .. lf inside the band
    for (int l = L - 1; l >= lf; --l) {
        const int np = 1 << l, s = 1 << (L - l);
        const int pr_y = d > 1 ? S / s : 1, pr_z = d > 2 ? S / s : 1;
        const int items = pr_y * pr_z * np;
        const long long *child = a.pyr + a.lvl_off[l + 1];
        long long *par = a.pyr + a.lvl_off[l];
        for (int t = tid; t < items; t += nt) {
            const int kx = t % np, q = t / np;
            const int ky = d > 1 ? by * pr_y + q % pr_y : 0;
            const int kz = d > 2 ? bz * pr_z + q / pr_y : 0;
            par[kx + (int64_t)np * (ky + (int64_t)np * kz)] = level_prefix_at(d, l, child, kx, ky, kz);
        }
        __syncthreads();
    }
    // (3) the band's part of the coarser levels (zeroed by k_absmax_parts)
    const int npf = 1 << lf;
    const long long *pf = a.pyr + a.lvl_off[lf] + (int64_t)npf * (by + (int64_t)npf * bz);
    for (int l = lf - 1; l >= 0; --l) {
        const int np = 1 << l, step = 1 << (lf - l);
        const int ky = by >> (lf - l), kz = bz >> (lf - l);
        unsigned long long *par = reinterpret_cast<unsigned long long *>(
            a.pyr + a.lvl_off[l] + (int64_t)np * (ky + (int64_t)np * kz));
        for (int kx = tid; kx < np; kx += nt)
            atomicAdd(par + kx, (unsigned long long)__ldcg(pf + (int64_t)(kx + 1) * step - 1));
    }
}

// ---------------------------------------------------------------------------
// Step 2 of the panel-by-panel form (Sec. 3 as written) in one launch after k_absmax_parts:
// one block per band (the leaf rows of one panel row of level lf = L - c) (1) quantises the
// band's leaf values, (2) sums the 2^d children of every panel of levels L-1 .. lf inside the
// band, and (3) adds the band's part of every coarser panel with 64-bit integer atomics (those
// levels were zeroed by k_absmax_parts).  Each panel then holds the integer sum of its leaves
// (exact, whatever the order in which the atomics land).
// ---------------------------------------------------------------------------
constexpr int STEP2_BAND_MAX = 2048;         // panels of the band's level-lf row kept in smem

__global__ void __launch_bounds__(1024) k_step2_panels(Step2Args a)
{
    __shared__ float s_w[32];
    const int nt = blockDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = nt / 32;
    float m = 0.f;
    for (int k = tid; k < a.nparts; k += nt) m = fmaxf(m, a.part[k]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) s_w[warp] = m;
    __syncthreads();
    m = 0.f;
    for (int w = 0; w < nw; ++w) m = fmaxf(m, s_w[w]);
    if (blockIdx.x == 0 && tid == 0) *a.mx = __float_as_uint(m);
    int sh = 62;
    if (m > 0.f) {
        int e1, e2;
        frexpf(m, &e1);
        frexpf((float)a.N, &e2);
        sh = 62 - e1 - e2;
    }
    const int n = a.n, d = a.d, L = a.L, lf = a.lf;
    const int S = 1 << a.c;
    const int bands_y = d > 1 ? n / S : 1;
    const int by = d > 1 ? (int)(blockIdx.x % bands_y) : 0;
    const int bz = d > 2 ? (int)(blockIdx.x / bands_y) : 0;
    const int rows_y = d > 1 ? S : 1, rows_z = d > 2 ? S : 1;
    long long *pyr = a.pyr;
    // (1) leaf values round(u b 2^sh)
    if (a.vec) {
        long long *leaf = pyr + a.lvl_off[L];
        const int64_t cnt4 = (int64_t)rows_y * rows_z * (n >> 2);
        for (int64_t t = tid; t < cnt4; t += nt) {
            const int64_t e = 4 * t;
            const int x = (int)(e % n), r = (int)(e / n);
            const int iy = by * rows_y + r % rows_y, iz = bz * rows_z + r / rows_y;
            const int64_t g = x + (int64_t)n * (iy + (int64_t)n * iz);
            const float4 uv = *reinterpret_cast<const float4 *>(a.u + g);
            const float4 bv = *reinterpret_cast<const float4 *>(a.b + g);
            longlong2 q0, q1;
            q0.x = __float2ll_rn(ldexpf(uv.x * bv.x, sh));
            q0.y = __float2ll_rn(ldexpf(uv.y * bv.y, sh));
            q1.x = __float2ll_rn(ldexpf(uv.z * bv.z, sh));
            q1.y = __float2ll_rn(ldexpf(uv.w * bv.w, sh));
            reinterpret_cast<longlong2 *>(leaf + g)[0] = q0;
            reinterpret_cast<longlong2 *>(leaf + g)[1] = q1;
        }
    } else {
        long long *leaf = pyr + a.lvl_off[L];
        const int64_t cnt = (int64_t)rows_y * rows_z * n;
        for (int64_t t = tid; t < cnt; t += nt) {
            const int x = (int)(t % n), r = (int)(t / n);
            const int iy = by * rows_y + r % rows_y, iz = bz * rows_z + r / rows_y;
            const int64_t g = x + (int64_t)n * (iy + (int64_t)n * iz);
            leaf[g] = __float2ll_rn(ldexpf(a.u[g] * a.b[g], sh));
        }
    }
    __syncthreads();
    // (2) levels L-1 .. lf inside the band
    for (int l = L - 1; l >= lf; --l) {
        const int np = 1 << l, s = 1 << (L - l), nc = 2 * np;
        const int pr_y = d > 1 ? S / s : 1, pr_z = d > 2 ? S / s : 1;
        const int items = pr_y * pr_z * np;
        const long long *child = pyr + a.lvl_off[l + 1];
        long long *par = pyr + a.lvl_off[l];
        for (int t = tid; t < items; t += nt) {
            const int kx = t % np, q = t / np;
            const int ky = d > 1 ? by * pr_y + q % pr_y : 0;
            const int kz = d > 2 ? bz * pr_z + q / pr_y : 0;
            long long v = 0;
            for (int c = 0; c < (1 << d); ++c) {
                const int cx = 2 * kx + (c & 1);
                const int cy = d > 1 ? 2 * ky + ((c >> 1) & 1) : 0;
                const int cz = d > 2 ? 2 * kz + ((c >> 2) & 1) : 0;
                v += __ldcg(child + cx + (int64_t)nc * (cy + (int64_t)nc * cz));
            }
            par[kx + (int64_t)np * (ky + (int64_t)np * kz)] = v;
        }
        __syncthreads();
    }
    // (3) the band's part of the coarser panels: the band's row of level lf is halved level by
    // level in shared memory (pairs of neighbours summed), each level's sums added to the
    // panels of that level with integer atomics
    if (lf == 0) return;
    const int npf = 1 << lf;
    const long long *pf = pyr + a.lvl_off[lf] + (int64_t)npf * (by + (int64_t)npf * bz);
    __shared__ long long s_band[STEP2_BAND_MAX];
    if (npf <= STEP2_BAND_MAX) {
        for (int k = tid; k < npf; k += nt) s_band[k] = __ldcg(pf + k);
        __syncthreads();
        for (int l = lf - 1; l >= 0; --l) {
            const int np = 1 << l;
            const int ky = by >> (lf - l), kz = bz >> (lf - l);
            unsigned long long *par = reinterpret_cast<unsigned long long *>(
                pyr + a.lvl_off[l] + (int64_t)np * (ky + (int64_t)np * kz));
            long long v[4];
            int cntv = 0;
            for (int kx = tid; kx < np; kx += nt) {     // read every pair before any write
                const long long w = s_band[2 * kx] + s_band[2 * kx + 1];
                if (cntv < 4) v[cntv] = w;
                ++cntv;
            }
            __syncthreads();
            cntv = 0;
            for (int kx = tid; kx < np; kx += nt, ++cntv) {
                s_band[kx] = v[cntv];
                atomicAdd(par + kx, (unsigned long long)v[cntv]);
            }
            __syncthreads();
        }
        return;
    }
    for (int l = lf - 1; l >= 0; --l) {
        const int np = 1 << l, step = 1 << (lf - l);
        const int ky = by >> (lf - l), kz = bz >> (lf - l);
        unsigned long long *par = reinterpret_cast<unsigned long long *>(
            pyr + a.lvl_off[l] + (int64_t)np * (ky + (int64_t)np * kz));
        for (int kx = tid; kx < np; kx += nt) {
            long long v = 0;
            for (int j = 0; j < step; ++j) v += __ldcg(pf + (int64_t)kx * step + j);
            atomicAdd(par + kx, (unsigned long long)v);
        }
    }
}

// ---------------------------------------------------------------------------
// Step 1 + Step 3 panel by panel (Sec. 3 as written, K = 0, integer route), 1-D and 2-D.
// Every distance the decomposition compares with the threshold is a half-unit gap 2t - 1
// between the node and a cell boundary (t >= 1 cells), or 0, so each node first tabulates its
// chords ch(t) = floor(sqrt(T4 - (2t - 1)^2)) (ch(0) = floor(sqrt(T4))) in shared memory --
// about R integer square roots -- and every level, panel row and parent row then reads its
// chord from the table.  Levels whose panels cannot fit in the ball are skipped, the parent
// row's fully-inside run is shared by its two child rows, and the panels of each run are added
// one by one from the pyramid.  The integer total equals that of k_fast_gather_i64.
// ---------------------------------------------------------------------------
constexpr int GP_THREADS = 128;
constexpr int GP_CHORDS = 24;

// gap index t of cell boundary c (cells) seen from node row iy: |2c - (2 iy + 1)| = 2t - 1
__device__ __forceinline__ int gap_t(int c, int iy) { return c > iy ? c - iy : iy - c + 1; }

template <int D>
__global__ void __launch_bounds__(GP_THREADS) k_fast_gather_panels_lane(FastI64Args a,
                                                                   const float *__restrict__ u,
                                                                   float *__restrict__ Lu)
{
    __shared__ int s_ch[GP_CHORDS * GP_THREADS];
    const int64_t i = blockIdx.x * (int64_t)GP_THREADS + threadIdx.x;
    if (i >= a.N) return;
    const int n = a.n, L = a.L;
    const int ix = (int)(i % n);
    const int iy = D > 1 ? (int)(i / n) : 0;
    const int X = 2 * ix + 1;
    const int T4 = a.thr4[i];
    const int r0 = isqrt_fast(T4);
    const int tmax = (r0 + 1) >> 1;          // (2t - 1)^2 <= T4 exactly for t <= tmax
    int *ch = s_ch + threadIdx.x;
    if (D > 1) {
        const int tc = min(tmax, GP_CHORDS - 1);
        ch[0] = r0;
        for (int t = 1; t <= tc; ++t) ch[t * GP_THREADS] = isqrt_fast(T4 - sq(2 * t - 1));
    }
    auto chord = [&](int t) -> int {
        if (D == 1) return r0;
        return t < GP_CHORDS ? ch[t * GP_THREADS] : isqrt_fast(T4 - sq(2 * t - 1));
    };
    int lmin = 0;
    while (lmin < L && (1 << (L - lmin + 1)) > 2 * r0) ++lmin;
    long long G = 0;
    for (int l = lmin; l <= L; ++l) {
        const int np = 1 << l;
        const int lg = L - l;                // panel side 2^lg cells, 2^(lg+1) half-units
        const int shf = lg + 1;
        const bool leaf = (l == L);
        const long long *__restrict__ lev = a.pyr + a.lvl_off[l];
        int ylo = 0, yhi = 0;
        if (D > 1) {
            if (leaf) {
                ylo = max(0, iy - tmax);
                yhi = min(n - 1, iy + tmax);
            } else {                         // rows whose far edges have t <= tmax
                ylo = max(0, -((tmax - 1 - iy) >> lg));
                yhi = min(np - 1, ((iy + tmax) >> lg) - 1);
            }
        }
        int pm = -1, ppa = 1, ppb = 0;
        for (int ky = ylo; ky <= yhi; ++ky) {
            int r;
            if (D == 1) r = r0;
            else if (leaf) r = chord(ky > iy ? ky - iy : iy - ky);
            else r = chord(max(gap_t(ky << lg, iy), gap_t((ky + 1) << lg, iy)));
            int ka, kb;
            if (leaf) {
                ka = max(0, -((r - X) >> 1) - 1);
                kb = min(n - 1, (X + r) >> 1);
            } else {
                ka = max(0, -((r - X) >> shf));
                kb = min(np - 1, ((X + r) >> shf) - 1);
            }
            if (ka > kb) continue;
            if (l > lmin && (ky >> 1) != pm) {       // the parent row's fully-inside run
                pm = ky >> 1;
                ppa = 1; ppb = 0;
                int tp = 0;
                if (D > 1) tp = max(gap_t(pm << (lg + 1), iy), gap_t((pm + 1) << (lg + 1), iy));
                if (tp <= tmax) {
                    const int rp = chord(tp);
                    const int qa = max(0, -((rp - X) >> (shf + 1)));
                    const int qb = min((np >> 1) - 1, ((X + rp) >> (shf + 1)) - 1);
                    if (qa <= qb) { ppa = 2 * qa; ppb = 2 * qb + 1; }
                }
            }
            const long long *__restrict__ row = lev + (int64_t)np * ky;
            const int b1 = ppa <= ppb ? min(kb, ppa - 1) : kb;
            for (int k = ka; k <= b1; ++k) G += __ldg(row + k);
            if (ppa <= ppb)
                for (int k = max(ka, ppb + 1); k <= kb; ++k) G += __ldg(row + k);
        }
    }
    const int sh = fixed_shift_f32(a.N, a.mx);
    Lu[i] = fixed_epilogue(G, u[i], a.selfQ[i], a.Fh[i], a.fastF[i], a.selfS[i], a.hd, sh);
}

// ---------------------------------------------------------------------------
// Step 1 stored (the decomposition of Algorithm 1 as set-up data, as the paper's timings
// treat it), warp-aligned.  The 32 nodes of a warp share their row (n >= 32) or the single
// row (1-D); the warp walks the union of its nodes' levels and panel rows, and every (level,
// panel row, side) of that walk in which some node has panels is one slot: the warp's
// smallest first-panel position in the pyramid buffer (one 32-bit word per warp and slot)
// and, per node, a 16-bit record (offset from that position: low byte; number of consecutive
// panels: high byte; 0 = none).  In a slot the nodes' panels are adjacent or shared, so a
// warp's loads of a slot touch few sectors.  The slots of a warp come in groups of four (the
// last group padded with empty slots: base 0, records 0), so that one 16-byte load gives a
// group's four base words and one 8-byte load a node's four records.  Layout per warp w, from
// its group offset woff[w], slot s = 4 g + k < wslots[w]: base[(woff + g) * 4 + k],
// rec[((woff + g) * 32 + lane) * 4 + k].
// ---------------------------------------------------------------------------

struct SlotArgs {
    int n, L;
    int64_t N;
    const int *thr4;
    int64_t lvl_off[NL_MAX_LEVELS + 2];
};

template <int D, bool WRITE>
__global__ void __launch_bounds__(GP_THREADS) k_slots(SlotArgs a, int *__restrict__ wslots,
                                                      const int64_t *__restrict__ woff,
                                                      unsigned *__restrict__ base,
                                                      unsigned short *__restrict__ rec,
                                                      int *__restrict__ bad)
{
    __shared__ int s_ch[GP_CHORDS * GP_THREADS];
    const int64_t i0 = blockIdx.x * (int64_t)GP_THREADS + threadIdx.x;
    const int64_t w = i0 >> 5;
    if ((w << 5) >= a.N) return;                      // whole warps only
    const int lane = threadIdx.x & 31;
    const bool act = i0 < a.N;
    const int64_t i = act ? i0 : a.N - 1;
    const int n = a.n, L = a.L;
    const int ix = (int)(i % n);
    const int iy = D > 1 ? (int)(i / n) : 0;
    const int X = 2 * ix + 1;
    const int T4 = a.thr4[i];
    const int r0 = isqrt_fast(T4);
    const int tmax = (r0 + 1) >> 1;
    int *ch = s_ch + threadIdx.x;
    if (D > 1) {
        const int tc = min(tmax, GP_CHORDS - 1);
        ch[0] = r0;
        for (int t = 1; t <= tc; ++t) ch[t * GP_THREADS] = isqrt_fast(T4 - sq(2 * t - 1));
    }
    auto chord = [&](int t) -> int {
        if (D == 1) return r0;
        return t < GP_CHORDS ? ch[t * GP_THREADS] : isqrt_fast(T4 - sq(2 * t - 1));
    };
    int lmin = 0;
    while (lmin < L && (1 << (L - lmin + 1)) > 2 * r0) ++lmin;
    const int lmin_w = __reduce_min_sync(0xffffffffu, lmin);
    const int tmax_w = __reduce_max_sync(0xffffffffu, tmax);
    const int64_t off = WRITE ? woff[w] : 0;
    int slot = 0, fault = 0;
    for (int l = lmin_w; l <= L; ++l) {
        const int np = 1 << l;
        const int lg = L - l;
        const int shf = lg + 1;
        const bool leaf = (l == L);
        int ylo = 0, yhi = 0;
        if (D > 1) {
            if (leaf) {
                ylo = max(0, iy - tmax_w);
                yhi = min(n - 1, iy + tmax_w);
            } else {
                ylo = max(0, -((tmax_w - 1 - iy) >> lg));
                yhi = min(np - 1, ((iy + tmax_w) >> lg) - 1);
            }
        }
        int pm = -1, ppa = 1, ppb = 0;
        for (int ky = ylo; ky <= yhi; ++ky) {
            int t = 0;
            if (D > 1)
                t = leaf ? (ky > iy ? ky - iy : iy - ky)
                         : max(gap_t(ky << lg, iy), gap_t((ky + 1) << lg, iy));
            int ka = 1, kb = 0;
            if (act && l >= lmin && t <= tmax) {
                const int r = chord(t);
                if (leaf) {
                    ka = max(0, -((r - X) >> 1) - 1);
                    kb = min(n - 1, (X + r) >> 1);
                } else {
                    ka = max(0, -((r - X) >> shf));
                    kb = min(np - 1, ((X + r) >> shf) - 1);
                }
            }
            if (l > lmin_w && (ky >> 1) != pm) {
                pm = ky >> 1;
                ppa = 1; ppb = 0;
                int tp = 0;
                if (D > 1) tp = max(gap_t(pm << (lg + 1), iy), gap_t((pm + 1) << (lg + 1), iy));
                if (act && l > lmin && tp <= tmax) {
                    const int rp = chord(tp);
                    const int qa = max(0, -((rp - X) >> (shf + 1)));
                    const int qb = min((np >> 1) - 1, ((X + rp) >> (shf + 1)) - 1);
                    if (qa <= qb) { ppa = 2 * qa; ppb = 2 * qb + 1; }
                }
            }
            const bool split = ppa <= ppb;
            const int b1 = split ? min(kb, ppa - 1) : kb;
            const int a2 = split ? max(ka, ppb + 1) : kb + 1;
            const int len[2] = { max(0, b1 - ka + 1), max(0, kb - a2 + 1) };
            const int st[2] = { ka, a2 };
            const int64_t rowpos = a.lvl_off[l] + (int64_t)np * ky;
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const unsigned pos = len[side] > 0 ? (unsigned)(rowpos + st[side]) : 0xffffffffu;
                const unsigned bmin = __reduce_min_sync(0xffffffffu, pos);
                if (bmin == 0xffffffffu) continue;           // no node of the warp: no slot
                if (WRITE) {
                    unsigned short r = 0;
                    if (len[side] > 0) {
                        const unsigned dlt = pos - bmin;
                        if (dlt > 255u || len[side] > 255) fault = 1;
                        r = (unsigned short)((dlt & 255u) | ((unsigned)min(len[side], 255) << 8));
                    }
                    rec[((off + (slot >> 2)) * 32 + lane) * 4 + (slot & 3)] = r;
                    if (lane == 0) base[off * 4 + slot] = bmin;
                }
                ++slot;
            }
        }
    }
    if (!WRITE && lane == 0) wslots[w] = slot;
    if (WRITE && fault) atomicExch(bad, 1);
}

// Step 3 from the stored slots, a group of four slots at a time: one broadcast 16-byte load of
// the group's base words, one 8-byte load of the node's four records, then the node's panels
// (the first SLOT_RUN_AHEAD of each run requested together, longer runs in a loop); the next
// group's words are requested before the current ones are used.
constexpr int SLOT_RUN_AHEAD = 3;     // panels of each run requested together (the vote in
                                      // slot_group tests length bytes >= 4 = SLOT_RUN_AHEAD + 1)
constexpr int SLOT_MIN_BLOCKS = 4;    // blocks of 256 per SM (64 registers, no spills)

__device__ __forceinline__ void slot_group(long long &G, const long long *__restrict__ pyr,
                                           const uint4 b, const uint2 q)
{
    constexpr int J = SLOT_RUN_AHEAD;
    static_assert(J == 3, "the long-run vote below tests length bytes >= 4");
    const unsigned bw[4] = { b.x, b.y, b.z, b.w };
    const unsigned rw[4] = { q.x & 0xffffu, q.x >> 16, q.y & 0xffffu, q.y >> 16 };
    long long v[4][J];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const long long *p = pyr + (bw[k] + (rw[k] & 255u));
        const int len = (int)(rw[k] >> 8);
#pragma unroll
        for (int j = 0; j < J; ++j) v[k][j] = j < len ? __ldg(p + j) : 0LL;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int j = 0; j < J; ++j) G += v[k][j];
    }
    // runs longer than J panels (a length byte >= 4): one warp vote per group
    if (__any_sync(0xffffffffu, ((q.x | q.y) & 0xFC00FC00u) != 0u)) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long *p = pyr + (bw[k] + (rw[k] & 255u));
            const int len = (int)(rw[k] >> 8);
            for (int j = J; j < len; ++j) G += __ldg(p + j);
        }
    }
}

__global__ void __launch_bounds__(256, SLOT_MIN_BLOCKS) k_fast_gather_slots(FastI64Args a,
                                                           const unsigned *__restrict__ base,
                                                           const unsigned short *__restrict__ rec,
                                                           const int64_t *__restrict__ woff,
                                                           const int *__restrict__ wslots,
                                                           const float *__restrict__ u,
                                                           float *__restrict__ Lu, int tiles_x)
{
    // tiles_x > 0 (2-D): the block's eight warps take the same 32 columns of eight consecutive
    // rows, so that their balls, and the pyramid panels they read, overlap in the SM's L1
    // (taller tiles of 16 and 32 rows were measured slower); tiles_x = 0: the warps of a block
    // take consecutive nodes
    const int lane = threadIdx.x & 31;
    int64_t w;
    if (tiles_x > 0)
        w = ((int64_t)(blockIdx.x / tiles_x) * 8 + (threadIdx.x >> 5)) * tiles_x +
            blockIdx.x % tiles_x;
    else
        w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t i = (w << 5) + lane;
    if ((w << 5) >= a.N) return;
    const int64_t off = woff[w];
    const int ng = (wslots[w] + 3) >> 2;
    const uint4 *__restrict__ b4 = reinterpret_cast<const uint4 *>(base) + off;
    const uint2 *__restrict__ q4 = reinterpret_cast<const uint2 *>(rec) + off * 32 + lane;
    const long long *__restrict__ pyr = a.pyr;
    long long G = 0;
    const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
    const uint2 z2 = make_uint2(0u, 0u);
    uint4 b = ng > 0 ? __ldg(b4) : z4;
    uint2 q = ng > 0 ? __ldcs(q4) : z2;
    for (int g = 0; g < ng; ++g) {
        const uint4 bn = g + 1 < ng ? __ldg(b4 + g + 1) : z4;
        const uint2 qn = g + 1 < ng ? __ldcs(q4 + (int64_t)(g + 1) * 32) : z2;
        slot_group(G, pyr, b, q);
        b = bn;
        q = qn;
    }
    if (i >= a.N) return;
    const int sh = fixed_shift_f32(a.N, a.mx);
    Lu[i] = fixed_epilogue(G, u[i], a.selfQ[i], a.Fh[i], a.fastF[i], a.selfS[i], a.hd, sh);
}

// Warp-uniform form for n >= 32 (the 32 nodes of a warp share their row): every lane walks
// the union of the warp's levels and panel rows, and each run's panels are added in a loop
// over the warp's longest run length with the shorter runs predicated off, so control flow
// never diverges; lane l reads panel ka_l + j, and the lanes' panels are adjacent or shared.
template <int D>
__global__ void __launch_bounds__(GP_THREADS) k_fast_gather_panels(FastI64Args a,
                                                                   const float *__restrict__ u,
                                                                   float *__restrict__ Lu)
{
    __shared__ int s_ch[GP_CHORDS * GP_THREADS];
    const int64_t i0 = blockIdx.x * (int64_t)GP_THREADS + threadIdx.x;
    const bool act = i0 < a.N;
    const int64_t i = act ? i0 : a.N - 1;
    const int n = a.n, L = a.L;
    const int ix = (int)(i % n);
    const int iy = D > 1 ? (int)(i / n) : 0;           // the same for the whole warp
    const int X = 2 * ix + 1;
    const int T4 = a.thr4[i];
    const int r0 = isqrt_fast(T4);
    const int tmax = (r0 + 1) >> 1;
    int *ch = s_ch + threadIdx.x;
    if (D > 1) {
        const int tc = min(tmax, GP_CHORDS - 1);
        ch[0] = r0;
        for (int t = 1; t <= tc; ++t) ch[t * GP_THREADS] = isqrt_fast(T4 - sq(2 * t - 1));
    }
    auto chord = [&](int t) -> int {
        if (D == 1) return r0;
        return t < GP_CHORDS ? ch[t * GP_THREADS] : isqrt_fast(T4 - sq(2 * t - 1));
    };
    int lmin = 0;
    while (lmin < L && (1 << (L - lmin + 1)) > 2 * r0) ++lmin;
    const int lmin_w = __reduce_min_sync(0xffffffffu, lmin);
    const int tmax_w = __reduce_max_sync(0xffffffffu, tmax);
    long long G = 0;
    for (int l = lmin_w; l <= L; ++l) {
        const int np = 1 << l;
        const int lg = L - l;
        const int shf = lg + 1;
        const bool leaf = (l == L);
        const long long *__restrict__ lev = a.pyr + a.lvl_off[l];
        int ylo = 0, yhi = 0;
        if (D > 1) {
            if (leaf) {
                ylo = max(0, iy - tmax_w);
                yhi = min(n - 1, iy + tmax_w);
            } else {
                ylo = max(0, -((tmax_w - 1 - iy) >> lg));
                yhi = min(np - 1, ((iy + tmax_w) >> lg) - 1);
            }
        }
        int pm = -1, ppa = 1, ppb = 0;
        for (int ky = ylo; ky <= yhi; ++ky) {
            int t = 0;
            if (D > 1)
                t = leaf ? (ky > iy ? ky - iy : iy - ky)
                         : max(gap_t(ky << lg, iy), gap_t((ky + 1) << lg, iy));
            int ka = 1, kb = 0;
            if (l >= lmin && t <= tmax) {
                const int r = chord(t);
                if (leaf) {
                    ka = max(0, -((r - X) >> 1) - 1);
                    kb = min(n - 1, (X + r) >> 1);
                } else {
                    ka = max(0, -((r - X) >> shf));
                    kb = min(np - 1, ((X + r) >> shf) - 1);
                }
            }
            if (l > lmin_w && (ky >> 1) != pm) {       // the parent row's fully-inside run
                pm = ky >> 1;
                ppa = 1; ppb = 0;
                int tp = 0;
                if (D > 1) tp = max(gap_t(pm << (lg + 1), iy), gap_t((pm + 1) << (lg + 1), iy));
                if (l > lmin && tp <= tmax) {
                    const int rp = chord(tp);
                    const int qa = max(0, -((rp - X) >> (shf + 1)));
                    const int qb = min((np >> 1) - 1, ((X + rp) >> (shf + 1)) - 1);
                    if (qa <= qb) { ppa = 2 * qa; ppb = 2 * qb + 1; }
                }
            }
            const bool split = ppa <= ppb;
            const int b1 = split ? min(kb, ppa - 1) : kb;
            const int a2 = split ? max(ka, ppb + 1) : kb + 1;
            const int len1 = max(0, b1 - ka + 1), len2 = max(0, kb - a2 + 1);
            const int m1 = __reduce_max_sync(0xffffffffu, len1);
            const int m2 = __reduce_max_sync(0xffffffffu, len2);
            const long long *__restrict__ row = lev + (int64_t)np * ky;
            for (int j = 0; j < m1; j += 2) {
                const long long v0 = j < len1 ? __ldg(row + ka + j) : 0LL;
                const long long v1 = j + 1 < len1 ? __ldg(row + ka + j + 1) : 0LL;
                G += v0 + v1;
            }
            for (int j = 0; j < m2; j += 2) {
                const long long v0 = j < len2 ? __ldg(row + a2 + j) : 0LL;
                const long long v1 = j + 1 < len2 ? __ldg(row + a2 + j + 1) : 0LL;
                G += v0 + v1;
            }
        }
    }
    if (!act) return;
    const int sh = fixed_shift_f32(a.N, a.mx);
    Lu[i] = fixed_epilogue(G, u[i], a.selfQ[i], a.Fh[i], a.fastF[i], a.selfS[i], a.hd, sh);
}

template <int D, typename T>
__global__ void __launch_bounds__(256) k_fast_gather_rowprefix(FastI64Args a,
                                                               const T *__restrict__ u,
                                                               T *__restrict__ Lu)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int n = a.n, L = a.L;
    const int ix = (int)(i % n);
    const int iy = D > 1 ? (int)((i / n) % n) : 0;
    const int iz = D > 2 ? (int)(i / ((int64_t)n * n)) : 0;
    const int X = 2 * ix + 1, Y = 2 * iy + 1, Z = 2 * iz + 1;
    const int T4 = a.thr4[i];
    const int r0 = isqrt_fast(T4);
    long long G = 0;
    // a panel of side 2^sh half-units fits in the ball only if 2^sh <= 2 r0
    int lmin = 0;
    while (lmin < L && (1 << (L - lmin + 1)) > 2 * r0) ++lmin;
    for (int l = lmin; l <= L; ++l) {
        const int np = 1 << l;
        const int sh = L - l + 1;
        const bool leaf = (l == L);
        const long long *lev = a.pyr + a.lvl_off[l];
        int ylo = 0, yhi = 0, zlo = 0, zhi = 0;
        if (D > 1) {
            ylo = max(0, -((r0 - Y) >> sh) - (leaf ? 1 : 0));
            yhi = min(np - 1, ((Y + r0) >> sh) - (leaf ? 0 : 1));
        }
        if (D > 2) {
            zlo = max(0, -((r0 - Z) >> sh) - (leaf ? 1 : 0));
            zhi = min(np - 1, ((Z + r0) >> sh) - (leaf ? 0 : 1));
        }
        for (int kz = zlo; kz <= zhi; ++kz) {
            const int z0 = (kz << sh) - Z, z1 = z0 + (1 << sh);
            const int ez = D > 2 ? (leaf ? (z0 > 0 ? sq(z0) : (z1 < 0 ? sq(z1) : 0))
                                         : max(sq(z0), sq(z1))) : 0;
            const int pz0 = ((kz >> 1) << (sh + 1)) - Z, pz1 = pz0 + (2 << sh);
            const int epz = D > 2 ? max(sq(pz0), sq(pz1)) : 0;
            int pm = -1, ppa = 1 << 30, ppb = -1;
            for (int ky = ylo; ky <= yhi; ++ky) {
                const int y0 = (ky << sh) - Y, y1 = y0 + (1 << sh);
                int e = ez;
                if (D > 1) e += leaf ? (y0 > 0 ? sq(y0) : (y1 < 0 ? sq(y1) : 0))
                                     : max(sq(y0), sq(y1));
                if (e > T4) continue;
                const int r = isqrt_fast(T4 - e);
                int ka, kb;
                if (leaf) {
                    ka = max(0, -((r - X) >> sh) - 1);
                    kb = min(np - 1, (X + r) >> sh);
                } else {
                    ka = max(0, -((r - X) >> sh));
                    kb = min(np - 1, ((X + r) >> sh) - 1);
                }
                // parent row's fully-inside panels (child units); shared by the two child rows
                if (l > 0 && (ky >> 1) != pm) {
                    pm = ky >> 1;
                    ppa = 1 << 30; ppb = -1;
                    const int py0 = (pm << (sh + 1)) - Y, py1 = py0 + (2 << sh);
                    const int ep = epz + (D > 1 ? max(sq(py0), sq(py1)) : 0);
                    if (ep <= T4) {
                        const int rp = isqrt_fast(T4 - ep);
                        const int qa = max(0, -((rp - X) >> (sh + 1)));
                        const int qb = min((np >> 1) - 1, ((X + rp) >> (sh + 1)) - 1);
                        if (qa <= qb) { ppa = 2 * qa; ppb = 2 * qb + 1; }
                    }
                }
                int pa = kb + 1, pb = kb;           // empty: beyond kb
                if (l > 0 && ppa <= ppb) { pa = ppa; pb = ppb; }
                const long long *row = lev + (int64_t)np * (ky + (int64_t)np * kz);
                // runs [ka, min(kb, pa-1)] and [max(ka, pb+1), kb], summed as prefix differences
                const int a1 = ka, b1 = min(kb, pa - 1);
                const int a2 = max(ka, pb + 1), b2 = kb;
                if (a1 <= b1) G += row[b1] - (a1 > 0 ? row[a1 - 1] : 0LL);
                if (a2 <= b2) G += row[b2] - (a2 > 0 ? row[a2 - 1] : 0LL);
            }
        }
    }
    const int sh = fixed_shift_f32(a.N, a.mx);
    Lu[i] = (T)fixed_epilogue(G, (float)u[i], a.selfQ[i], a.Fh[i], a.fastF[i], a.selfS[i], a.hd, sh);
}

// ---------------------------------------------------------------------------
// Leaf-row form of Step 3 (K = 0, integer route).  The panels of Algorithm 1 tile exactly the
// leaf cells that meet the open ball, so their sum is, row by row, the run of leaf cells of
// that row that meets the ball: one difference of the leaf-row prefix sums per row.  The
// integer total is the one the panel-by-panel and per-level routes add.  Rows iy + t and
// iy - t (and likewise in z) have the same vertical gap, so they share one chord.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long leaf_run(const long long *__restrict__ row, int n, int X,
                                              int r)
{
    const int ka = max(0, -((r - X) >> 1) - 1);
    const int kb = min(n - 1, (X + r) >> 1);
    return __ldg(row + kb) - (ka > 0 ? __ldg(row + ka - 1) : 0LL);
}

template <int D>
__device__ __forceinline__ long long leaf_plane(const long long *__restrict__ plane, int n,
                                                int X, int iy, int T4)
{
    if (D == 1) return leaf_run(plane, n, X, isqrt_fast(T4));
    long long G = 0;
    for (int t = 0;; ++t) {
        const int e = t == 0 ? 0 : sq(2 * t - 1);
        if (e > T4) break;
        const int r = isqrt_fast(T4 - e);
        if (iy + t < n) G += leaf_run(plane + (int64_t)n * (iy + t), n, X, r);
        if (t > 0 && iy - t >= 0) G += leaf_run(plane + (int64_t)n * (iy - t), n, X, r);
    }
    return G;
}

template <int D, typename T>
__global__ void __launch_bounds__(256) k_fast_gather_leafrows(FastI64Args a,
                                                              const T *__restrict__ u,
                                                              T *__restrict__ Lu)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int n = a.n;
    const int ix = (int)(i % n);
    const int iy = D > 1 ? (int)((i / n) % n) : 0;
    const int iz = D > 2 ? (int)(i / ((int64_t)n * n)) : 0;
    const int X = 2 * ix + 1;
    const int T4 = a.thr4[i];
    const long long *leaf = a.pyr + a.lvl_off[a.L];
    long long G = 0;
    if (D < 3) {
        G = leaf_plane<D>(leaf, n, X, iy, T4);
    } else {
        const int64_t pl = (int64_t)n * n;
        for (int t = 0;; ++t) {
            const int ez = t == 0 ? 0 : sq(2 * t - 1);
            if (ez > T4) break;
            if (iz + t < n) G += leaf_plane<2>(leaf + pl * (iz + t), n, X, iy, T4 - ez);
            if (t > 0 && iz - t >= 0) G += leaf_plane<2>(leaf + pl * (iz - t), n, X, iy, T4 - ez);
        }
    }
    const int sh = fixed_shift_f32(a.N, a.mx);
    Lu[i] = (T)fixed_epilogue(G, (float)u[i], a.selfQ[i], a.Fh[i], a.fastF[i], a.selfS[i], a.hd, sh);
}

// ---------------------------------------------------------------------------
// Step 2 of the leaf rows for several right-hand sides in three launches (rows of 128 or 256
// nodes, 16-byte aligned fields): per-block bounds of |u| for every right-hand side, their
// reduction to one scale word per right-hand side, then one warp per leaf row reading the
// coefficient b once and every right-hand side's u, each scanned lane-contiguously (as the
// single right-hand-side path) and stored through shared memory.  Every prefix is the integer
// the single right-hand-side route writes.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_absmax_parts_multi(int64_t N, const float *__restrict__ u,
                                                            float bmax, unsigned char *aux,
                                                            int stride)
{
    __shared__ float s_w[8];
    const int q = blockIdx.y;
    const float *__restrict__ uq = u + (int64_t)q * N;
    float m = 0.f;
    const int64_t stride_t = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const float4 *__restrict__ u4 = reinterpret_cast<const float4 *>(uq);
    const int64_t N4 = N >> 2;                        // N is a multiple of 4 here
    for (int64_t i = t0; i < N4; i += 8 * stride_t) {
        float4 x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t j = i + k * stride_t;
            x[k] = j < N4 ? u4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
            m = fmaxf(fmaxf(m, fmaxf(fabsf(x[k].x), fabsf(x[k].y))),
                      fmaxf(fabsf(x[k].z), fabsf(x[k].w)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmaxf(m, s_w[w]);
        float *part = reinterpret_cast<float *>(aux + (size_t)q * stride + 16);
        part[blockIdx.x] = (m * bmax) * (1.f + 0x1p-20f);
    }
}

// one block per right-hand side: the bound word (first word of its aux) from the parts
__global__ void __launch_bounds__(256) k_parts_reduce(unsigned char *aux, int stride, int nparts)
{
    __shared__ float s_w[8];
    unsigned char *a = aux + (size_t)blockIdx.x * stride;
    const float *part = reinterpret_cast<const float *>(a + 16);
    float m = 0.f;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) m = fmaxf(m, part[k]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmaxf(m, s_w[w]);
        *reinterpret_cast<unsigned int *>(a) = __float_as_uint(m);
    }
}

struct Step2MultiArgs {
    int d, n, c, count, stride;
    int64_t N;
    const float *u, *b;
    const unsigned char *aux;
    long long *leaf;                 // [count][N]
};

__global__ void __launch_bounds__(128) k_step2_leaf_multi(Step2MultiArgs a)
{
    __shared__ long long s_row[4 * 256];
    __shared__ int s_sh[LEAF_MULTI_MAX];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (tid < a.count) {
        const unsigned int *mx = reinterpret_cast<const unsigned int *>(a.aux + (size_t)tid * a.stride);
        s_sh[tid] = fixed_shift_f32(a.N, mx);
    }
    __syncthreads();
    const int n = a.n, d = a.d, E = n / 32;
    const int S = 1 << a.c;
    const int bands_y = d > 1 ? n / S : 1;
    const int by = d > 1 ? (int)(blockIdx.x % bands_y) : 0;
    const int bz = d > 2 ? (int)(blockIdx.x / bands_y) : 0;
    const int rows_y = d > 1 ? S : 1, rows_z = d > 2 ? S : 1;
    long long *srow = s_row + warp * n;
    for (int r = warp; r < rows_y * rows_z; r += nw) {
        const int iy = by * rows_y + r % rows_y, iz = bz * rows_z + r / rows_y;
        const int64_t row = (int64_t)n * (iy + (int64_t)n * iz);
        const float4 *__restrict__ b4 = reinterpret_cast<const float4 *>(a.b + row) + lane * (E / 4);
        float bv[8];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (4 * k < E) {
                const float4 y = b4[k];
                bv[4 * k] = y.x; bv[4 * k + 1] = y.y; bv[4 * k + 2] = y.z; bv[4 * k + 3] = y.w;
            }
        }
        for (int q = 0; q < a.count; ++q) {
            const int sh = s_sh[q];
            const float4 *__restrict__ u4 =
                reinterpret_cast<const float4 *>(a.u + (int64_t)q * a.N + row) + lane * (E / 4);
            float v[8];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (4 * k < E) {
                    const float4 x = u4[k];
                    v[4 * k] = x.x * bv[4 * k]; v[4 * k + 1] = x.y * bv[4 * k + 1];
                    v[4 * k + 2] = x.z * bv[4 * k + 2]; v[4 * k + 3] = x.w * bv[4 * k + 3];
                }
            }
            long long qv[8], t = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (k < E) {
                    t += __float2ll_rn(ldexpf(v[k], sh));
                    qv[k] = t;
                }
            }
            const long long off = warp_incl_scan_ll(t, lane) - t;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (k < E) srow[E * lane + k] = qv[k] + off;
            __syncwarp();
            long long *out = a.leaf + (int64_t)q * a.N + row;
            for (int x = lane; x < n; x += 32) out[x] = srow[x];
            __syncwarp();
        }
    }
}

// Several right-hand sides at once (leaf-row form): the run bounds of a row are computed once
// and applied to every right-hand side's leaf-row prefix sums (leaf + r * N, scale mx[r]).

constexpr int AUX_STRIDE = 16 + NL_FAST_PARTS * 4;     // bytes of one right-hand side's aux

struct LeafMultiArgs {
    int n, count;
    int64_t N;
    const int *thr4;
    const double *fastF, *selfS, *selfQ;
    const float *Fh;
    const long long *leaf;               // [count][N]
    const unsigned char *aux;            // [count][AUX_STRIDE], max |v| in the first word
    double hd;
};

template <int D>
__device__ __forceinline__ void leaf_runs_multi(long long (&G)[LEAF_MULTI], const long long *leaf,
                                                int64_t N, int count, int64_t rowoff, int n,
                                                int X, int r)
{
    const int ka = max(0, -((r - X) >> 1) - 1);
    const int kb = min(n - 1, (X + r) >> 1);
#pragma unroll
    for (int q = 0; q < LEAF_MULTI; ++q) {
        if (q < count) {
            const long long *row = leaf + (int64_t)q * N + rowoff;
            G[q] += __ldg(row + kb) - (ka > 0 ? __ldg(row + ka - 1) : 0LL);
        }
    }
}

template <int D, typename T>
__global__ void __launch_bounds__(256) k_fast_gather_leafrows_multi(LeafMultiArgs a,
                                                                    const T *__restrict__ u,
                                                                    T *__restrict__ Lu)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int n = a.n;
    const int ix = (int)(i % n);
    const int iy = D > 1 ? (int)((i / n) % n) : 0;
    const int iz = D > 2 ? (int)(i / ((int64_t)n * n)) : 0;
    const int X = 2 * ix + 1;
    const int T4 = a.thr4[i];
    long long G[LEAF_MULTI];
#pragma unroll
    for (int q = 0; q < LEAF_MULTI; ++q) G[q] = 0;
    if (D == 1) {
        leaf_runs_multi<D>(G, a.leaf, a.N, a.count, 0, n, X, isqrt_fast(T4));
    } else {
        const int64_t pl = (int64_t)n * n;
        for (int tz = 0; tz <= (D > 2 ? n : 0); ++tz) {
            const int ez = tz == 0 ? 0 : sq(2 * tz - 1);
            if (ez > T4) break;
            for (int sz = 0; sz < (D > 2 && tz > 0 ? 2 : 1); ++sz) {
                const int z = D > 2 ? (sz ? iz - tz : iz + tz) : 0;
                if (z < 0 || z >= (D > 2 ? n : 1)) continue;
                const int64_t zoff = pl * z;
                for (int ty = 0;; ++ty) {
                    const int e = ez + (ty == 0 ? 0 : sq(2 * ty - 1));
                    if (e > T4) break;
                    const int r = isqrt_fast(T4 - e);
                    if (iy + ty < n)
                        leaf_runs_multi<D>(G, a.leaf, a.N, a.count, zoff + (int64_t)n * (iy + ty), n, X, r);
                    if (ty > 0 && iy - ty >= 0)
                        leaf_runs_multi<D>(G, a.leaf, a.N, a.count, zoff + (int64_t)n * (iy - ty), n, X, r);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < LEAF_MULTI; ++q) {
        if (q < a.count) {
            const unsigned int *mx = (const unsigned int *)(a.aux + (size_t)q * AUX_STRIDE);
            const int sh = fixed_shift_f32(a.N, mx);
            const int64_t g = (int64_t)q * a.N + i;
            Lu[g] = (T)fixed_epilogue(G[q], (float)u[g], a.selfQ[i], a.Fh[i], a.fastF[i],
                                      a.selfS[i], a.hd, sh);
        }
    }
}

// Leaf rows in 3-D for a constant horizon (every node's leaf set has the same shape): a block
// of 32 x 8 x 4 outputs (a thread takes one (x, y) and four z) stages, per right-hand side, the
// leaf-row prefix sums of every row its outputs reach -- (8 + 2 TM) x (4 + 2 TM) rows of
// 32 + 2 TM + 1 values, x clamped as the run bounds clamp them (0 before the first cell, the
// last prefix past the end), rows outside the grid as zeros -- in shared memory with
// asynchronous copies, then adds each output's rows as two shared-memory reads.  TM is both
// the row reach (rows |ty|, |tz| <= TM) and the longest run ((isqrt(T4) + 1) / 2 cells each
// side), so the tile geometry and every row's position in it are compile-time constants; only
// a row's run length c (its chord, -1 outside the ball) is read, once for the four z-outputs.
// The integers are those of k_fast_gather_leafrows_multi: the same runs, exact sums.
constexpr int R3_BX = 32, R3_BY = 8, R3_BZ = 4;
constexpr int R3_TM_MAX = 8;

struct Rows3Args {
    int n, count;
    int64_t N;
    const long long *leaf;            // [count][N] leaf-row prefix sums
    const unsigned char *aux;         // per right-hand side the scale word, aux_stride apart
    int aux_stride;
    const double *fastF, *selfS, *selfQ;
    const float *Fh;
    double hd;
    int T4;                           // the common threshold (half units)
};

template <int TM>
__global__ void __launch_bounds__(256) k_fast_gather_rows3c(Rows3Args a, const float *__restrict__ u,
                                                            float *__restrict__ Lu)
{
    constexpr int SXX = R3_BX + 2 * TM + 1, SYY = R3_BY + 2 * TM, SZZ = R3_BZ + 2 * TM;
    constexpr int W = 2 * TM + 1;
    extern __shared__ __align__(16) long long s3[];
    __shared__ int s_c[W * W];                        // run half-length per (tz, ty), -1: none
    const int n = a.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = blockIdx.x * R3_BX, y0 = blockIdx.y * R3_BY, z0 = blockIdx.z * R3_BZ;
    for (int k = tid; k < W * W; k += 256) {
        const int tz = k / W - TM, ty = k % W - TM;
        const int e = (tz == 0 ? 0 : (2 * abs(tz) - 1) * (2 * abs(tz) - 1)) +
                      (ty == 0 ? 0 : (2 * abs(ty) - 1) * (2 * abs(ty) - 1));
        s_c[k] = e <= a.T4 ? (isqrt_fast(a.T4 - e) + 1) >> 1 : -1;
    }
    const int x = x0 + lane, y = y0 + warp;
    const long long *centre = s3 + (TM * SYY + warp + TM) * SXX + lane + TM + 1;   // (x, y, z0)
    for (int q = 0; q < a.count; ++q) {
        const long long *__restrict__ P = a.leaf + (int64_t)q * a.N;
        __syncthreads();                          // the chords, or the last tile, are done
        // one warp per staged row, lanes along x; asynchronous 8-byte copies (zero-filled
        // outside the grid and before the first cell), all in flight before the one wait
        for (int rz = warp; rz < SYY * SZZ; rz += 8) {
            const int yy = rz % SYY, zz = rz / SYY;
            const int gy = y0 - TM + yy, gz = z0 - TM + zz;
            long long *dst = s3 + rz * SXX;
            const bool inside = gy >= 0 && gy < n && gz >= 0 && gz < n;
            const long long *src = inside ? P + (int64_t)n * (gy + (int64_t)n * gz) : P;
#pragma unroll
            for (int xx = lane; xx < SXX; xx += 32) {
                const int gx = x0 - TM - 1 + xx;
                const bool ok = inside && gx >= 0;
                const unsigned d = (unsigned)__cvta_generic_to_shared(dst + xx);
                const long long *g = ok ? src + min(gx, n - 1) : P;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;"
                             ::"r"(d), "l"(g), "r"(ok ? 8 : 0) : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        long long G[R3_BZ];
#pragma unroll
        for (int zo = 0; zo < R3_BZ; ++zo) G[zo] = 0;
#pragma unroll
        for (int tz = -TM; tz <= TM; ++tz) {
#pragma unroll
            for (int ty = -TM; ty <= TM; ++ty) {
                const int c = s_c[(tz + TM) * W + ty + TM];
                if (c >= 0) {
                    const long long *row = centre + (tz * SYY + ty) * SXX;
                    const long long *hi = row + c, *lo = row - c - 1;
#pragma unroll
                    for (int zo = 0; zo < R3_BZ; ++zo)
                        G[zo] += hi[zo * SYY * SXX] - lo[zo * SYY * SXX];
                }
            }
        }
        const unsigned int *mx = (const unsigned int *)(a.aux + (size_t)q * a.aux_stride);
        const int sh = fixed_shift_f32(a.N, mx);
#pragma unroll
        for (int zo = 0; zo < R3_BZ; ++zo) {
            const int z = z0 + zo;
            if (x < n && y < n && z < n) {
                const int64_t i = x + (int64_t)n * (y + (int64_t)n * z);
                const int64_t g = (int64_t)q * a.N + i;
                Lu[g] = fixed_epilogue(G[zo], u[g], a.selfQ[i], a.Fh[i], a.fastF[i], a.selfS[i],
                                       a.hd, sh);
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static size_t rows3_smem(int tm);

static int moments_count(int d, int K)
{
    int M = 0;
    for (int a2 = 0; a2 <= (d > 2 ? 2 * K : 0); ++a2)
        for (int a1 = 0; a1 <= (d > 1 ? 2 * K : 0); ++a1)
            for (int a0 = 0; a0 <= 2 * K; ++a0)
                if (a0 + a1 + a2 <= 2 * K) ++M;
    return M;
}

// Step 1 at plan time for the panel-by-panel route (1-D with n >= 32, and 2-D with n >= 32):
// count every warp's slots, offsets on the host, write the slots.  Skipped (the gather then
// enumerates the decomposition itself) when pyramid positions need more than 32 bits, the
// slots would exceed 2^23 (about 570 MB), or a node's offset or run length leaves its byte.
static nl_status build_slots(nl_plan *p, cudaStream_t st)
{
    const int64_t N = p->N;
    if (p->lvl_off[p->L] + N >= ((int64_t)1 << 32) - 256) return NL_OK;
    SlotArgs sa;
    sa.n = p->n; sa.L = p->L; sa.N = N; sa.thr4 = p->thr4;
    for (int l = 0; l <= p->L; ++l) sa.lvl_off[l] = p->lvl_off[l];
    const int64_t nw = (N + 31) / 32;
    int *wslots = nullptr, *bad = nullptr;
    int64_t *woff = nullptr;
    unsigned *base = nullptr;
    unsigned short *rec = nullptr;
    auto fail = [&](nl_status s) {
        if (wslots) cudaFree(wslots);
        if (bad) cudaFree(bad);
        if (woff) cudaFree(woff);
        if (base) cudaFree(base);
        if (rec) cudaFree(rec);
        return s;
    };
    if (cudaMalloc(&wslots, nw * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&woff, nw * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&bad, sizeof(int)) != cudaSuccess) {
        nl_set_error("nl_plan_create: allocation for the stored decomposition failed");
        return fail(NL_ENOMEM);
    }
    const unsigned g = (unsigned)((nw * 32 + GP_THREADS - 1) / GP_THREADS);
    if (p->d == 1) k_slots<1, false><<<g, GP_THREADS, 0, st>>>(sa, wslots, woff, base, rec, bad);
    else k_slots<2, false><<<g, GP_THREADS, 0, st>>>(sa, wslots, woff, base, rec, bad);
    std::vector<int> hw(nw);
    std::vector<int64_t> ho(nw);
    cudaError_t ce = cudaMemcpyAsync(hw.data(), wslots, nw * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return fail(nl_cuda_fail(ce, "stored decomposition (counts)"));
    int64_t groups = 0;                   // groups of four slots (woff counts groups)
    for (int64_t w = 0; w < nw; ++w) { ho[w] = groups; groups += (hw[w] + 3) / 4; }
    const int64_t tot = 4 * groups;
    if (tot > ((int64_t)1 << 23)) return fail(NL_OK);
    const size_t base_bytes = std::max<int64_t>(tot, 4) * sizeof(unsigned);
    const size_t rec_bytes = std::max<int64_t>(tot, 4) * 32 * sizeof(unsigned short);
    if (cudaMalloc(&base, base_bytes) != cudaSuccess || cudaMalloc(&rec, rec_bytes) != cudaSuccess) {
        nl_set_error("nl_plan_create: allocation of %lld decomposition slots failed", (long long)tot);
        return fail(NL_ENOMEM);
    }
    ce = cudaMemsetAsync(bad, 0, sizeof(int), st);
    // the padding slots of each warp's last group stay empty
    if (ce == cudaSuccess) ce = cudaMemsetAsync(base, 0, base_bytes, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(rec, 0, rec_bytes, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(woff, ho.data(), nw * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) return fail(nl_cuda_fail(ce, "stored decomposition (offsets)"));
    if (p->d == 1) k_slots<1, true><<<g, GP_THREADS, 0, st>>>(sa, wslots, woff, base, rec, bad);
    else k_slots<2, true><<<g, GP_THREADS, 0, st>>>(sa, wslots, woff, base, rec, bad);
    int hb = 0;
    ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return fail(nl_cuda_fail(ce, "stored decomposition (slots)"));
    if (hb) return fail(NL_OK);
    cudaFree(bad);
    p->slot_base = base;
    p->slot_rec = rec;
    p->slot_woff = woff;
    p->slot_count = wslots;
    p->slots = (size_t)tot;
    p->device_bytes += (size_t)tot * (sizeof(unsigned) + 32 * sizeof(unsigned short)) +
                       nw * (sizeof(int) + sizeof(int64_t));
    return NL_OK;
}

nl_status nl_fast_plan_init(nl_plan *p, const double *delta_dev, const double *a_dev,
                            cudaStream_t st)
{
    const int d = p->d, K = p->K, L = p->L;
    // fast path unavailable (apply reports NL_EUNSUPPORTED): n not a power of two, or
    // n > 8192 (integer half-unit geometry is kept within 32 bits)
    if (L < 0 || p->n > 8192) return NL_OK;
    p->M = moments_count(d, K);
    const int M = p->M;
    // multi-indices in the compact order (a2 outer, a1, a0 inner)
    std::vector<int> al;
    for (int a2 = 0; a2 <= (d > 2 ? 2 * K : 0); ++a2)
        for (int a1 = 0; a1 <= (d > 1 ? 2 * K : 0); ++a1)
            for (int a0 = 0; a0 <= 2 * K; ++a0)
                if (a0 + a1 + a2 <= 2 * K) { al.push_back(a0); al.push_back(a1); al.push_back(a2); }
    // re-centring: child s in {0,1}^d, t_parent = (t_child + 2 s - 1) / 2, so
    // t_p^alpha = prod_k 2^{-alpha_k} sum_{beta_k} C(alpha_k, beta_k) (2s_k - 1)^{alpha_k - beta_k} t_c^{beta_k}
    std::vector<double> shift((size_t)(1 << d) * M * M, 0.0);
    auto binom = [](int a, int b) {
        double r = 1.0;
        for (int t = 0; t < b; ++t) r = r * (a - t) / (t + 1);
        return r;
    };
    for (int s = 0; s < (1 << d); ++s)
        for (int ia = 0; ia < M; ++ia)
            for (int ib = 0; ib < M; ++ib) {
                double c = 1.0;
                for (int k = 0; k < d && c != 0.0; ++k) {
                    const int A = al[3 * ia + k], Bb = al[3 * ib + k];
                    if (Bb > A) { c = 0.0; break; }
                    const double sg = ((s >> k) & 1) ? 1.0 : -1.0;
                    c *= binom(A, Bb) * std::pow(sg, A - Bb) * std::ldexp(1.0, -A);
                }
                shift[((size_t)s * M + ia) * M + ib] = c;
            }
    int64_t off = 0;
    for (int l = 0; l < L; ++l) {
        p->lvl_off[l] = off;
        int64_t P = 1;
        for (int q = 0; q < d; ++q) P *= ((int64_t)1 << l);
        off += P * M;
    }
    off = (off + 1) & ~(int64_t)1; // leaf level 16-byte aligned
    p->lvl_off[L] = off;           // leaf level: N values of v
    const int64_t total = off + p->N;

    auto alloc = [&](void **ptr, size_t bytes) -> nl_status {
        cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 1);
        if (e != cudaSuccess) {
            nl_set_error("cudaMalloc(%zu) for the fast path: %s", bytes, cudaGetErrorString(e));
            return NL_ENOMEM;
        }
        p->device_bytes += bytes;
        return NL_OK;
    };
    nl_status s;
    if ((s = alloc((void **)&p->pyr, total * sizeof(double))) != NL_OK) return s;
    if ((s = alloc((void **)&p->shift, shift.size() * sizeof(double))) != NL_OK) return s;
    if ((s = alloc((void **)&p->malpha, al.size() * sizeof(int))) != NL_OK) return s;
    if ((s = alloc((void **)&p->fastF, p->N * sizeof(double))) != NL_OK) return s;
    if ((s = alloc((void **)&p->selfS, p->N * sizeof(double))) != NL_OK) return s;
    if ((s = alloc((void **)&p->ir4, p->N * sizeof(double))) != NL_OK) return s;
    // K >= 1, d <= 2: the integer leaf-row route (prefix arrays of k^e q, e <= 2K); 2^bits
    // bounds a node's exact sums: (2 Rmax + 3)^d cells times (Rmax + 1)^{2K}
    const double kint_bound = std::pow(2.0 * p->Rmax + 3.0, (double)d) *
                              std::pow(p->Rmax + 1.0, 2.0 * K);
    const bool kint = K >= 1 && d <= 2 && kint_bound <= 0x1p40;
    if (K == 0 || kint) {
        const size_t aux = 16 + NL_FAST_PARTS * sizeof(float);
        if ((s = alloc((void **)&p->fast_mx, aux)) != NL_OK) return s;
        NL_CUDA_TRY(cudaMemsetAsync(p->fast_mx, 0, aux, st));     // the ticket starts at 0
        if ((s = alloc((void **)&p->selfQ, p->N * sizeof(double))) != NL_OK) return s;
        if ((s = alloc((void **)&p->fastFh32, p->N * sizeof(float))) != NL_OK) return s;
    }
    if (kint) {
        if ((s = alloc((void **)&p->kint_P, (size_t)(2 * K + 1) * p->N * sizeof(long long))) != NL_OK)
            return s;
        p->kint_bits = (int)std::ceil(std::log2(kint_bound));
    }
    double *d_pc = nullptr;
    if ((s = alloc((void **)&d_pc, 8 * sizeof(double))) != NL_OK) return s;
    NL_CUDA_TRY(cudaMemcpyAsync(p->shift, shift.data(), shift.size() * sizeof(double),
                                cudaMemcpyHostToDevice, st));
    NL_CUDA_TRY(cudaMemcpyAsync(p->malpha, al.data(), al.size() * sizeof(int),
                                cudaMemcpyHostToDevice, st));
    NL_CUDA_TRY(cudaMemcpyAsync(d_pc, p->poly, 8 * sizeof(double), cudaMemcpyHostToDevice, st));
    const double pi = 3.141592653589793238462643383279502884;
    const double sphere = d == 1 ? 2.0 : (d == 2 ? 2.0 * pi : 4.0 * pi);
    const unsigned gb = (unsigned)((p->N + 255) / 256);
    k_fast_node<<<gb, 256, 0, st>>>(d, p->n, K, p->coef, p->self_mode, p->N, p->sigma, sphere,
                                    delta_dev, a_dev, p->thr4, d_pc, p->fastF, p->selfS, p->ir4);
    NL_CUDA_TRY(cudaGetLastError());
    if (K == 0 || kint) {
        k_fixed_consts<<<gb, 256, 0, st>>>(p->N, std::pow(p->h, (double)d), p->fastF, p->selfS,
                                           p->selfQ, p->fastFh32);
        // the plan-time bound max |b| of the fixed-point scale (word 2 of the aux header)
        unsigned int *bw = reinterpret_cast<unsigned int *>(p->fast_mx) + 2;
        const unsigned gm = (unsigned)std::min<int64_t>((p->N + 255) / 256, 1024);
        k_max_abs_bits<<<gm, 256, 0, st>>>(p->N, p->b32, bw);
        unsigned int bits = 0;
        NL_CUDA_TRY(cudaMemcpyAsync(&bits, bw, sizeof(bits), cudaMemcpyDeviceToHost, st));
        NL_CUDA_TRY(cudaStreamSynchronize(st));
        memcpy(&p->fast_bmax, &bits, sizeof(float));
    }
    if (K == 0) {
        // 3-D, constant horizon: the common threshold and the staged gather's tile geometry
        p->r3_tm = 0;
        if (d == 3 && p->const_horizon) {
            int T4 = -1;
            NL_CUDA_TRY(cudaMemcpy(&T4, p->thr4, sizeof(int), cudaMemcpyDeviceToHost));
            // rows |t| <= tm with (2t - 1)^2 <= T4, runs of at most (isqrt(T4) + 1) / 2 cells
            // each side: the same bound
            int r0 = 0;
            while ((r0 + 1) * (r0 + 1) <= T4) ++r0;
            const int tm = (r0 + 1) >> 1;
            if (T4 >= 1 && tm >= 1 && tm <= R3_TM_MAX && rows3_smem(tm) <= 160 * 1024) {
                p->r3_T4 = T4;
                p->r3_tm = tm;
            }
        }
    }
    NL_CUDA_TRY(cudaGetLastError());
    NL_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(d_pc);
    p->device_bytes -= 8 * sizeof(double);
    if (K == 0 && p->fast_variant == NL_FAST_PANELS && d <= 2 && p->n >= 32)
        return build_slots(p, st);
    return NL_OK;
}

// tracing: event k (0: before Step 2, 1: before Step 3, 2: after Step 3) of this apply
static void prof_mark(nl_plan *p, int k, cudaStream_t st)
{
    if (!p->prof_on || p->prof_count >= 64) return;
    cudaEvent_t &e = p->prof_ev[p->prof_count][k];
    if (!e && cudaEventCreate(&e) != cudaSuccess) { e = nullptr; return; }
    cudaEventRecord(e, st);
    if (k == 2) p->prof_count++;
}

// Step 2 of the row-prefix form: per-block bounds (and the coarse levels zeroed), then one
// fused build (see k_step2_rowprefix).  The band side 2^c is 16 leaf rows in 2-D and 8 per
// axis in 3-D (capped by the grid); in 1-D the single row is the band.
static cudaError_t step2_rowprefix(nl_plan *p, const float *u, bool leaf_only, cudaStream_t st,
                                   long long *leaf_out = nullptr, unsigned char *aux = nullptr)
{
    const int d = p->d, L = p->L;
    long long *pyr = (long long *)p->pyr;
    if (!aux) aux = (unsigned char *)p->fast_mx;
    unsigned int *mx = (unsigned int *)aux;
    float *part = (float *)(aux + 16);
    int64_t per = (p->N + NL_FAST_PARTS - 1) / NL_FAST_PARTS;
    if (per < 2048) per = 2048;
    const int nparts = (int)((p->N + per - 1) / per);
    // bands: one panel row of level lf = L - c; the leaf rows alone need no levels, so they
    // take bands of four rows (a warp each) for more blocks
    int c = 0;
    if (d == 2) c = std::min(leaf_only ? 2 : 4, L);
    if (d == 3) c = std::min(leaf_only ? 1 : 3, L);
    // the leaf rows alone of 2-D or 1-D grids with n >= 512: n / 256 warps per row, 16 / wpr
    // rows (at least one) per block
    int wpr = 1;
    if (leaf_only && d <= 2 && p->n >= 512) {
        wpr = p->n / 256;
        const int rb = std::max(1, 16 / wpr);
        c = 0;
        while (d == 2 && (1 << (c + 1)) <= rb) ++c;
    }
    int rows = 1;
    for (int q = 1; q < d; ++q) rows <<= c;
    const int threads = leaf_only ? std::max(32, std::min(1024, 32 * rows * wpr)) : STEP2_THREADS;
    Step2Args a;
    a.d = d; a.n = p->n; a.L = L; a.c = c; a.lf = L - c; a.N = p->N;
    a.u = u; a.b = p->b32; a.part = part; a.nparts = nparts;
    a.mx = mx; a.pyr = pyr; a.leaf_only = leaf_only ? 1 : 0; a.wpr = wpr;
    a.lane_e = 0; a.vec = 0;
    {
        int rows_blk = 1;
        for (int q = 1; q < d; ++q) rows_blk <<= c;
        if (leaf_only && wpr == 1 && rows_blk <= 4 && (p->n == 128 || p->n == 256) &&
            ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(p->b32)) & 15) == 0)
            a.lane_e = p->n / 32;
    }
    a.leaf = leaf_out ? leaf_out : pyr + p->lvl_off[L];
    for (int l = 0; l <= L; ++l) a.lvl_off[l] = p->lvl_off[l];
    k_absmax_parts<<<nparts, 256, 0, st>>>(p->N, u, p->fast_bmax, part, pyr,
                                           leaf_only ? 0 : p->lvl_off[a.lf]);
    int64_t bands = 1;
    for (int q = 1; q < d; ++q) bands *= p->n >> c;
    k_step2_rowprefix<<<(unsigned)bands, threads, 0, st>>>(a);
    return cudaGetLastError();
}

// Step 2 of the panel-by-panel form: per-block bounds (and the coarse levels zeroed), then one
// fused build of every level (k_step2_panels).  Bands of 4 leaf rows in 2-D, 8 x 8 in 3-D; in
// 1-D the single row is the band.
static cudaError_t step2_panels(nl_plan *p, const float *u, cudaStream_t st)
{
    const int d = p->d, L = p->L;
    long long *pyr = (long long *)p->pyr;
    unsigned char *aux = (unsigned char *)p->fast_mx;
    float *part = (float *)(aux + 16);
    int64_t per = (p->N + NL_FAST_PARTS - 1) / NL_FAST_PARTS;
    if (per < 2048) per = 2048;
    const int nparts = (int)((p->N + per - 1) / per);
    int c = 0;
    if (d == 2) c = std::min(2, L);
    if (d == 3) c = std::min(3, L);
    Step2Args a;
    a.d = d; a.n = p->n; a.L = L; a.c = c; a.lf = L - c; a.N = p->N;
    a.u = u; a.b = p->b32; a.part = part; a.nparts = nparts;
    a.mx = (unsigned int *)aux; a.pyr = pyr; a.leaf_only = 0; a.wpr = 1; a.lane_e = 0;
    a.leaf = pyr + p->lvl_off[L];
    a.vec = (p->n % 4 == 0 &&
             ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(p->b32) |
               reinterpret_cast<uintptr_t>(a.leaf)) & 15) == 0) ? 1 : 0;
    for (int l = 0; l <= L; ++l) a.lvl_off[l] = p->lvl_off[l];
    k_absmax_parts<<<nparts, 256, 0, st>>>(p->N, u, p->fast_bmax, part, pyr, p->lvl_off[a.lf]);
    int64_t bands = 1;
    for (int q = 1; q < d; ++q) bands *= p->n >> c;
    k_step2_panels<<<(unsigned)bands, 512, 0, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Leaf-row form of the fast apply for K >= 1 (integer route, FP32 data, d <= 2; a deviation of
// the f1 kind from the FP64 moment pyramid, with the same leaf-set sum).  Along a leaf row of
// node i (row offset o_y) the weight is p(|o|^2 / R_i^2) = sum_m beta_m (o_y^2 + o_x^2)^m,
// beta_m = p_m / R_i^{2m}, so the row needs the run sums C_{2j} = sum_run o_x^{2j} q,
// o_x = k - i_x, j <= K: from prefix sums of k^e q (e <= 2K, modulo 2^64) by differences,
// centred by the binomial expansion.  They are accumulated, times o_y^{2(m-j)}, into the
// exact sums Z[m][j] (modulo 2^64; the true values are bounded by 2^bits max|q| < 2^61), and
// once per node G = sum_m beta_m sum_j binom(m, j) Z[m][j] 2^-S in FP64.  q = round(u b 2^S)
// as in the K = 0 route.
// ---------------------------------------------------------------------------
struct KintArgs {
    int n, bits, nparts;
    int64_t N;
    const float *u, *b, *part;
    unsigned int *mx;                 // max |u b| bound (FP32 bits), written by the scan
    long long *P;                     // [2K+1][N]
    const int *thr4;
    const double *fastF, *selfS, *ir4;
    double hd;
    double p[8];
};

__device__ __forceinline__ int kint_shift(const KintArgs &a, float m)
{
    if (!(m > 0.f)) return 61 - a.bits;
    int e1;
    frexpf(m, &e1);
    return 61 - a.bits - e1;
}

// one warp per leaf row: the 2K + 1 prefix arrays of k^e q (modulo 2^64)
template <int K>
__global__ void __launch_bounds__(128) k_kint_scan(KintArgs a)
{
    __shared__ float s_m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {
        float m = 0.f;
        for (int k = lane; k < a.nparts; k += 32) m = fmaxf(m, a.part[k]);
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_m = m;
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.mx = __float_as_uint(s_m);
    const int sh = kint_shift(a, s_m);
    const int n = a.n;
    const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + warp;
    if (row * n >= a.N) return;
    const int64_t base = row * n;
    typedef unsigned long long u64;
    u64 carry[2 * K + 1];
#pragma unroll
    for (int e = 0; e <= 2 * K; ++e) carry[e] = 0ull;
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int k = k0 + lane;
        u64 v[2 * K + 1];
        if (k < n) {
            const u64 q = (u64)__float2ll_rn(ldexpf(a.u[base + k] * a.b[base + k], sh));
            v[0] = q;
#pragma unroll
            for (int e = 1; e <= 2 * K; ++e) v[e] = v[e - 1] * (u64)k;
        } else {
#pragma unroll
            for (int e = 0; e <= 2 * K; ++e) v[e] = 0ull;
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int e = 0; e <= 2 * K; ++e) {
                const u64 w = __shfl_up_sync(0xffffffffu, v[e], o);
                if (lane >= o) v[e] += w;
            }
        }
#pragma unroll
        for (int e = 0; e <= 2 * K; ++e) {
            v[e] += carry[e];
            if (k < n) a.P[(int64_t)e * a.N + base + k] = (long long)v[e];
            carry[e] = __shfl_sync(0xffffffffu, v[e], 31);
        }
    }
}

template <int D, int K>
__global__ void __launch_bounds__(256) k_kint_gather(KintArgs a, float *__restrict__ Lu)
{
    typedef unsigned long long u64;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int n = a.n;
    const int ix = (int)(i % n);
    const int iy = D > 1 ? (int)(i / n) : 0;
    const int X = 2 * ix + 1;
    const int T4 = a.thr4[i];
    const int64_t N = a.N;
    u64 nk[2 * K + 1];                               // (-i_x)^e
    nk[0] = 1ull;
#pragma unroll
    for (int e = 1; e <= 2 * K; ++e) nk[e] = nk[e - 1] * (u64)(-(long long)ix);
    u64 Z[K + 1][K + 1];
#pragma unroll
    for (int m = 0; m <= K; ++m)
#pragma unroll
        for (int j = 0; j <= K; ++j) Z[m][j] = 0ull;
    for (int t = 0;; ++t) {
        const int e0 = t == 0 ? 0 : (2 * t - 1) * (2 * t - 1);
        if (e0 > T4 || (D == 1 && t > 0)) break;
        const int r = isqrt_fast(T4 - e0);
        const int ka = max(0, -((r - X) >> 1) - 1);
        const int kb = min(n - 1, (X + r) >> 1);
        for (int s = 0; s < (t > 0 ? 2 : 1); ++s) {
            const int dy = s ? -t : t;
            const int ky = iy + dy;
            if (ky < 0 || ky >= (D > 1 ? n : 1)) continue;
            const int64_t row = (int64_t)ky * n;
            u64 Dd[2 * K + 1];
#pragma unroll
            for (int e = 0; e <= 2 * K; ++e) {
                const long long *Pe = a.P + (int64_t)e * N + row;
                Dd[e] = (u64)__ldg(Pe + kb) - (ka > 0 ? (u64)__ldg(Pe + ka - 1) : 0ull);
            }
            u64 C[K + 1];                            // sum_run (k - i_x)^{2j} q
#pragma unroll
            for (int j = 0; j <= K; ++j) {
                u64 acc = 0ull, bin = 1ull;          // binom(2j, e), e = 0 ..
#pragma unroll
                for (int e = 0; e <= 2 * j; ++e) {
                    acc += bin * nk[2 * j - e] * Dd[e];
                    bin = bin * (u64)(2 * j - e) / (u64)(e + 1);
                }
                C[j] = acc;
            }
            const u64 dy2 = (u64)(long long)(dy * dy);
            u64 dyp[K + 1];
            dyp[0] = 1ull;
#pragma unroll
            for (int q = 1; q <= K; ++q) dyp[q] = dyp[q - 1] * dy2;
#pragma unroll
            for (int m = 0; m <= K; ++m)
#pragma unroll
                for (int j = 0; j <= m; ++j) Z[m][j] += dyp[m - j] * C[j];
        }
    }
    const int sh = kint_shift(a, __uint_as_float(*a.mx));
    const double ir2 = 4.0 * a.ir4[i];               // 1 / R_i^2
    double G = 0.0, beta = 1.0;
#pragma unroll
    for (int m = 0; m <= K; ++m) {
        double zm = 0.0, bin = 1.0;
#pragma unroll
        for (int j = 0; j <= m; ++j) {
            zm += bin * (double)(long long)Z[m][j];
            bin = bin * (m - j) / (j + 1);
        }
        G += a.p[m] * beta * zm;
        beta *= ir2;
    }
    G = ldexp(G, -sh);
    Lu[i] = (float)(a.fastF[i] * (a.hd * G - (double)a.u[i] * a.selfS[i]));
}

static nl_status fast_one_kint(nl_plan *p, const float *u, float *Lu, cudaStream_t st)
{
    prof_mark(p, 0, st);
    const int64_t N = p->N;
    unsigned char *aux = (unsigned char *)p->fast_mx;
    float *part = (float *)(aux + 16);
    int64_t per = (N + NL_FAST_PARTS - 1) / NL_FAST_PARTS;
    if (per < 2048) per = 2048;
    const int nparts = (int)((N + per - 1) / per);
    KintArgs a;
    a.n = p->n; a.bits = p->kint_bits; a.nparts = nparts; a.N = N;
    a.u = u; a.b = p->b32; a.part = part; a.mx = (unsigned int *)aux; a.P = p->kint_P;
    a.thr4 = p->thr4; a.fastF = p->fastF; a.selfS = p->selfS; a.ir4 = p->ir4;
    a.hd = std::pow(p->h, (double)p->d);
    for (int m = 0; m < 8; ++m) a.p[m] = p->poly[m];
    k_absmax_parts<<<nparts, 256, 0, st>>>(N, u, p->fast_bmax, part, nullptr, 0);
    const int64_t rows = N / p->n;
    const unsigned gs = (unsigned)((rows + 3) / 4), gb = (unsigned)((N + 255) / 256);
    switch (p->K) {
        case 1: k_kint_scan<1><<<gs, 128, 0, st>>>(a); break;
        case 2: k_kint_scan<2><<<gs, 128, 0, st>>>(a); break;
        default: k_kint_scan<3><<<gs, 128, 0, st>>>(a); break;
    }
    prof_mark(p, 1, st);
#define NL_KINT(D, KK) k_kint_gather<D, KK><<<gb, 256, 0, st>>>(a, Lu)
    if (p->d == 1) {
        if (p->K == 1) NL_KINT(1, 1); else if (p->K == 2) NL_KINT(1, 2); else NL_KINT(1, 3);
    } else {
        if (p->K == 1) NL_KINT(2, 1); else if (p->K == 2) NL_KINT(2, 2); else NL_KINT(2, 3);
    }
#undef NL_KINT
    prof_mark(p, 2, st);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

// the staged 3-D gather for a constant horizon (k_fast_gather_rows3c) where the plan set it up
static size_t rows3_smem(int tm)
{
    return sizeof(long long) * (size_t)(R3_BX + 2 * tm + 1) * (R3_BY + 2 * tm) * (R3_BZ + 2 * tm);
}

static bool rows3_usable(const nl_plan *p)
{
    return p->d == 3 && p->r3_tm > 0 && p->n % R3_BX == 0;
}

template <int TM>
static nl_status launch_rows3_t(const nl_plan *p, const Rows3Args &a, const float *u, float *Lu,
                                cudaStream_t st)
{
    const size_t smem = rows3_smem(TM);
    NL_CUDA_TRY(cudaFuncSetAttribute(k_fast_gather_rows3c<TM>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const dim3 grd((unsigned)(p->n / R3_BX), (unsigned)(p->n / R3_BY), (unsigned)(p->n / R3_BZ));
    k_fast_gather_rows3c<TM><<<grd, 256, smem, st>>>(a, u, Lu);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

static nl_status launch_rows3(nl_plan *p, const long long *leaf, const unsigned char *aux,
                              int aux_stride, int count, const float *u, float *Lu,
                              cudaStream_t st)
{
    Rows3Args a;
    a.n = p->n; a.count = count; a.N = p->N;
    a.leaf = leaf; a.aux = aux; a.aux_stride = aux_stride;
    a.fastF = p->fastF; a.selfS = p->selfS; a.selfQ = p->selfQ; a.Fh = p->fastFh32;
    a.hd = std::pow(p->h, 3.0);
    a.T4 = p->r3_T4;
    switch (p->r3_tm) {
    case 1: return launch_rows3_t<1>(p, a, u, Lu, st);
    case 2: return launch_rows3_t<2>(p, a, u, Lu, st);
    case 3: return launch_rows3_t<3>(p, a, u, Lu, st);
    case 4: return launch_rows3_t<4>(p, a, u, Lu, st);
    case 5: return launch_rows3_t<5>(p, a, u, Lu, st);
    case 6: return launch_rows3_t<6>(p, a, u, Lu, st);
    case 7: return launch_rows3_t<7>(p, a, u, Lu, st);
    default: return launch_rows3_t<8>(p, a, u, Lu, st);
    }
}

static nl_status fast_one_i64(nl_plan *p, const float *u, float *Lu, cudaStream_t st)
{
    prof_mark(p, 0, st);
    const int d = p->d, L = p->L;
    long long *pyr = (long long *)p->pyr;           // same buffer, 8-byte entries (M = 1)
    unsigned int *mx = (unsigned int *)p->fast_mx;
    const unsigned gb = (unsigned)((p->N + 255) / 256);
    const bool panels = p->fast_variant == NL_FAST_PANELS;
    if (panels) NL_CUDA_TRY(step2_panels(p, u, st));
    const bool prefix = !panels;
    const bool leafrows = p->fast_variant == NL_FAST_LEAFROWS;
    if (prefix) {
        NL_CUDA_TRY(step2_rowprefix(p, u, leafrows, st));
    }
    FastI64Args a;
    a.n = p->n; a.L = L; a.N = p->N;
    a.thr4 = p->thr4; a.fastF = p->fastF; a.selfS = p->selfS;
    a.selfQ = p->selfQ; a.Fh = p->fastFh32;
    a.pyr = pyr;
    for (int l = 0; l <= L; ++l) a.lvl_off[l] = p->lvl_off[l];
    a.hd = std::pow(p->h, (double)d);
    a.mx = mx;
    prof_mark(p, 1, st);
    if (leafrows) {
        if (d == 1) k_fast_gather_leafrows<1, float><<<gb, 256, 0, st>>>(a, u, Lu);
        else if (d == 2) k_fast_gather_leafrows<2, float><<<gb, 256, 0, st>>>(a, u, Lu);
        else if (rows3_usable(p)) {
            const nl_status s3 = launch_rows3(p, pyr + p->lvl_off[L], (const unsigned char *)mx,
                                              0, 1, u, Lu, st);
            if (s3 != NL_OK) return s3;
        } else k_fast_gather_leafrows<3, float><<<gb, 256, 0, st>>>(a, u, Lu);
    } else if (prefix) {
        if (d == 1) k_fast_gather_rowprefix<1, float><<<gb, 256, 0, st>>>(a, u, Lu);
        else if (d == 2) k_fast_gather_rowprefix<2, float><<<gb, 256, 0, st>>>(a, u, Lu);
        else k_fast_gather_rowprefix<3, float><<<gb, 256, 0, st>>>(a, u, Lu);
    } else {
        const unsigned gp = (unsigned)((p->N + GP_THREADS - 1) / GP_THREADS);
        if (p->slot_base) {
            const unsigned gr = (unsigned)(((p->N + 31) / 32 * 32 + 255) / 256);
            const int tiles_x = (d == 2 && p->n % 32 == 0) ? p->n / 32 : 0;
            k_fast_gather_slots<<<gr, 256, 0, st>>>(a, p->slot_base, p->slot_rec, p->slot_woff,
                                                     p->slot_count, u, Lu, tiles_x);
        } else if (d == 1) k_fast_gather_panels_lane<1><<<gp, GP_THREADS, 0, st>>>(a, u, Lu);
        else if (d == 2 && p->n >= 32) k_fast_gather_panels<2><<<gp, GP_THREADS, 0, st>>>(a, u, Lu);
        else if (d == 2) k_fast_gather_panels_lane<2><<<gp, GP_THREADS, 0, st>>>(a, u, Lu);
        else k_fast_gather_i64<3, float><<<gb, 256, 0, st>>>(a, u, Lu);
    }
    prof_mark(p, 2, st);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

template <typename T>
static nl_status fast_one(nl_plan *p, const T *u, T *Lu, cudaStream_t st)
{
    if (sizeof(T) == 4 && p->K == 0 && p->fast_mx && p->fast_variant != NL_FAST_FP64_PANELS)
        return fast_one_i64(p, (const float *)u, (float *)Lu, st);
    if (sizeof(T) == 4 && p->K >= 1 && p->kint_P && p->fast_variant == NL_FAST_LEAFROWS)
        return fast_one_kint(p, (const float *)u, (float *)Lu, st);
    prof_mark(p, 0, st);
    const int d = p->d, L = p->L, M = p->M;
    double *leaf = p->pyr + p->lvl_off[L];
    const unsigned gb = (unsigned)((p->N + 255) / 256);
    k_pyr_leaf<T><<<gb, 256, 0, st>>>(p->N, u, p->b64, leaf);
    for (int l = L - 1; l >= 0; --l) {
        int64_t P = 1;
        for (int q = 0; q < d; ++q) P *= ((int64_t)1 << l);
        const double *child = (l + 1 == L) ? leaf : p->pyr + p->lvl_off[l + 1];
        const unsigned g = (unsigned)((P + 127) / 128);
        k_pyr_level<<<g, 128, 0, st>>>(d, l, L, M, child, p->pyr + p->lvl_off[l], p->shift);
    }
    FastArgs a;
    a.d = d; a.n = p->n; a.L = L; a.K = p->K; a.M = M; a.N = p->N;
    a.thr4 = p->thr4; a.fastF = p->fastF; a.selfS = p->selfS; a.ir4 = p->ir4;
    a.pyr = p->pyr; a.leaf = leaf;
    for (int l = 0; l <= L; ++l) a.lvl_off[l] = p->lvl_off[l];
    a.hd = std::pow(p->h, (double)d);
    for (int m = 0; m < 8; ++m) a.poly[m] = p->poly[m];
    prof_mark(p, 1, st);
#define NL_GATHER(D, KK) k_fast_gather<D, KK, T><<<gb, 256, 0, st>>>(a, u, Lu)
    if (d == 1) {
        switch (p->K) { case 0: NL_GATHER(1, 0); break; case 1: NL_GATHER(1, 1); break;
                        case 2: NL_GATHER(1, 2); break; default: NL_GATHER(1, 3); }
    } else if (d == 2) {
        switch (p->K) { case 0: NL_GATHER(2, 0); break; case 1: NL_GATHER(2, 1); break;
                        case 2: NL_GATHER(2, 2); break; default: NL_GATHER(2, 3); }
    } else {
        switch (p->K) { case 0: NL_GATHER(3, 0); break; case 1: NL_GATHER(3, 1); break;
                        case 2: NL_GATHER(3, 2); break; default: NL_GATHER(3, 3); }
    }
#undef NL_GATHER
    prof_mark(p, 2, st);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

extern "C" nl_status nl_plan_profile(nl_plan *p, int enable)
{
    if (!nl_plan_ok(p)) {
        nl_set_error("nl_plan_profile: invalid plan");
        return NL_EINVAL;
    }
    p->prof_on = enable ? 1 : 0;
    p->prof_count = 0;
    return NL_OK;
}

extern "C" nl_status nl_plan_profile_read(nl_plan *p, double *step2_ms, double *step3_ms,
                                          int *applies)
{
    if (!nl_plan_ok(p) || !step2_ms || !step3_ms || !applies) {
        nl_set_error("nl_plan_profile_read: bad argument");
        return NL_EINVAL;
    }
    double s2 = 0.0, s3 = 0.0;
    for (int k = 0; k < p->prof_count; ++k) {
        float a = 0.f, b = 0.f;
        NL_CUDA_TRY(cudaEventSynchronize(p->prof_ev[k][2]));
        NL_CUDA_TRY(cudaEventElapsedTime(&a, p->prof_ev[k][0], p->prof_ev[k][1]));
        NL_CUDA_TRY(cudaEventElapsedTime(&b, p->prof_ev[k][1], p->prof_ev[k][2]));
        s2 += a;
        s3 += b;
    }
    *step2_ms = s2;
    *step3_ms = s3;
    *applies = p->prof_count;
    p->prof_count = 0;
    return NL_OK;
}

// several FP32 right-hand sides through the leaf-row route: Step 2 per right-hand side into
// its own leaf buffer, then one gather for up to LEAF_MULTI of them
static nl_status fast_multi_leafrows(nl_plan *p, const float *u, float *Lu, int nrhs,
                                     cudaStream_t st)
{
    const int G = std::min(nrhs, LEAF_MULTI);
    if (p->leaf_multi_cap < G) {
        if (p->leaf_multi) cudaFree(p->leaf_multi);
        if (p->aux_multi) cudaFree(p->aux_multi);
        p->leaf_multi = nullptr; p->aux_multi = nullptr; p->leaf_multi_cap = 0;
        if (cudaMalloc(&p->leaf_multi, (size_t)G * p->N * sizeof(long long)) != cudaSuccess ||
            cudaMalloc(&p->aux_multi, (size_t)G * AUX_STRIDE) != cudaSuccess) {
            nl_set_error("nl_apply_fast: allocation of %d leaf buffers failed", G);
            return NL_ENOMEM;
        }
        p->leaf_multi_cap = G;
    }
    const unsigned gb = (unsigned)((p->N + 255) / 256);
    for (int r0 = 0; r0 < nrhs; r0 += LEAF_MULTI) {
        const int cnt = std::min(LEAF_MULTI, nrhs - r0);
        prof_mark(p, 0, st);
        const float *u0 = u + (int64_t)r0 * p->N;
        const bool fused = p->d > 1 && (p->n == 128 || p->n == 256) &&
                           ((reinterpret_cast<uintptr_t>(u0) |
                             reinterpret_cast<uintptr_t>(p->b32)) & 15) == 0;
        if (fused) {
            int64_t per = (p->N + NL_FAST_PARTS - 1) / NL_FAST_PARTS;
            if (per < 2048) per = 2048;
            const int nparts = (int)((p->N + per - 1) / per);
            k_absmax_parts_multi<<<dim3(nparts, cnt), 256, 0, st>>>(p->N, u0, p->fast_bmax,
                                                                    p->aux_multi, AUX_STRIDE);
            k_parts_reduce<<<cnt, 256, 0, st>>>(p->aux_multi, AUX_STRIDE, nparts);
            Step2MultiArgs sa;
            sa.d = p->d; sa.n = p->n; sa.c = std::min(p->d == 2 ? 2 : 1, p->L);
            sa.count = cnt; sa.stride = AUX_STRIDE; sa.N = p->N;
            sa.u = u0; sa.b = p->b32; sa.aux = p->aux_multi; sa.leaf = p->leaf_multi;
            int64_t bands = 1;
            for (int q = 1; q < p->d; ++q) bands *= p->n >> sa.c;
            int rows = 1;
            for (int q = 1; q < p->d; ++q) rows <<= sa.c;
            k_step2_leaf_multi<<<(unsigned)bands, 32 * rows, 0, st>>>(sa);
            NL_CUDA_TRY(cudaGetLastError());
        } else {
            for (int q = 0; q < cnt; ++q)
                NL_CUDA_TRY(step2_rowprefix(p, u0 + (int64_t)q * p->N, true, st,
                                            p->leaf_multi + (int64_t)q * p->N,
                                            p->aux_multi + (size_t)q * AUX_STRIDE));
        }
        prof_mark(p, 1, st);
        LeafMultiArgs a;
        a.n = p->n; a.count = cnt; a.N = p->N;
        a.thr4 = p->thr4; a.fastF = p->fastF; a.selfS = p->selfS;
        a.selfQ = p->selfQ; a.Fh = p->fastFh32;
        a.leaf = p->leaf_multi; a.aux = p->aux_multi;
        a.hd = std::pow(p->h, (double)p->d);
        const float *ur = u + (int64_t)r0 * p->N;
        float *lr = Lu + (int64_t)r0 * p->N;
        if (p->d == 1) k_fast_gather_leafrows_multi<1, float><<<gb, 256, 0, st>>>(a, ur, lr);
        else if (p->d == 2) k_fast_gather_leafrows_multi<2, float><<<gb, 256, 0, st>>>(a, ur, lr);
        else if (rows3_usable(p)) {
            const nl_status s3 = launch_rows3(p, p->leaf_multi, p->aux_multi, AUX_STRIDE, cnt,
                                              ur, lr, st);
            if (s3 != NL_OK) return s3;
        } else k_fast_gather_leafrows_multi<3, float><<<gb, 256, 0, st>>>(a, ur, lr);
        NL_CUDA_TRY(cudaGetLastError());
        prof_mark(p, 2, st);
    }
    return NL_OK;
}

nl_status nl_fast_launch(nl_plan *p, const void *u, void *Lu, int nrhs, int dtype,
                         cudaStream_t st)
{
    if (nrhs > 1 && dtype == NL_F32 && p->K == 0 && p->fast_mx &&
        p->fast_variant == NL_FAST_LEAFROWS)
        return fast_multi_leafrows(p, (const float *)u, (float *)Lu, nrhs, st);
    for (int r = 0; r < nrhs; ++r) {
        nl_status s;
        if (dtype == NL_F32)
            s = fast_one<float>(p, (const float *)u + (int64_t)r * p->N, (float *)Lu + (int64_t)r * p->N, st);
        else
            s = fast_one<double>(p, (const double *)u + (int64_t)r * p->N, (double *)Lu + (int64_t)r * p->N, st);
        if (s != NL_OK) return s;
    }
    return NL_OK;
}

extern "C" nl_status nl_apply_fast(nl_plan *p, const void *u, void *Lu, int nrhs, int dtype,
                                   void *stream)
{
    if (!nl_plan_ok(p)) {
        nl_set_error("nl_apply_fast: invalid plan");
        return NL_EINVAL;
    }
    if (!u || !Lu || nrhs < 1 || (dtype != NL_F32 && dtype != NL_F64)) {
        nl_set_error("nl_apply_fast: need non-null u/Lu, nrhs >= 1, dtype F32/F64");
        return NL_EINVAL;
    }
    if (p->family == NL_PD_BOND) {
        if (dtype != NL_F32) {
            nl_set_error("nl_apply_fast: the fast peridynamic path takes FP32 data");
            return NL_EUNSUPPORTED;
        }
        return nl_fast_pd_launch(p, (const float *)u, (float *)Lu, nrhs, nl_stream(stream));
    }
    if (p->family != NL_POLY || p->symmetric || p->L < 0 || !p->pyr) {
        nl_set_error("nl_apply_fast: needs an NL_POLY plan (one-sided, or symmetric with "
                     "K <= 3) on n = 2^L <= 8192");
        return NL_EUNSUPPORTED;
    }
    if (p->self_mode == NL_SELF_PAPER && p->coef == NL_COEF_XY) {
        nl_set_error("nl_apply_fast: NL_SELF_PAPER is not defined for NL_COEF_XY");
        return NL_EUNSUPPORTED;
    }
    if (p->sym_fast) return nl_fast_sym_launch(p, u, Lu, nrhs, dtype, nl_stream(stream));
    return nl_fast_launch(p, u, Lu, nrhs, dtype, nl_stream(stream));
}
