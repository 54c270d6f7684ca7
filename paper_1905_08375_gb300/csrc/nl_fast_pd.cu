// nl_fast_pd.cu -- fast-path peridynamics of degree 0 (the outlook of Sec. 4: a fast
// algorithm for the linear peridynamic operator).  The bond tensor xi xi^T / |xi|^3 of
// Eq. (1.2) is replaced by xi xi^T p(|xi|/delta_i) / delta_i^3 with p = 1 (the degree-0
// member of the p^{2K} family, matched at the horizon), summed over the leaf set of
// Algorithm 1 -- every leaf cell meeting the open ball, inside Omega or not (outside:
// u = 0, c = c_i).  In lattice offsets o (xi = o h):
//   (L u)_i = F_i [ c_i A_i + B_i - M_i u_i ],   F_i = sigma h^{d+2} / (2 delta_i^3)
//   A_i = sum_{k in LS(i), in Omega} o o^T u_k,   B_i = the same with (c u)_k,
//   M_i = sum_{k in LS(i)} (c_i + c_k) o o^T      (plan-time constant, FP64).
// A and B are exact integer sums: each of u_x, u_y, c u_x, c u_y is rounded once to a
// multiple of 2^-S (S per field and apply, from its max |.|), and along every leaf row the
// prefix sums of q, k q and k^2 q (k the column) give, for the run of a row, the sums of q,
// k q and k^2 q by differences.  The prefix sums wrap modulo 2^64 (only differences over
// runs of at most 2R + 3 cells are used, and those fit); S is chosen so that, with C the
// bound (2R + 3)^2 on a leaf set's cells, n^2 C max|q| < 2^61: every per-node sum of
// differences (over rows, times dy or dy^2) and the final combination with the node's column
// (o_x = k - kx) then fit in 64-bit integers.  Rows and runs are those of the scalar leaf-row
// gather (the same half-unit geometry).  2-D, FP32 data.  K = 1, 2 (the polynomial
// micromodulus p^{2K} matched to s^-3) extend this below with the moments of o_x up to 2K + 2,
// and the 3-D form (K = 0) follows them.
#include <cmath>
#include <cstring>
#include <vector>

#include "nl_internal.cuh"

namespace {

constexpr int FPD_FIELDS = 4;                   // u_x, u_y, c u_x, c u_y
constexpr int FPD_ARRAYS = 10;                  // ux: P0 P1 P2, uy: P0 P1, cux: P0 P1 P2, cuy: P0 P1
constexpr int FPD_PARTS = 1024;

struct FpdPoly { double p[8]; };                // p_0 .. p_K of the micromodulus polynomial

__device__ __forceinline__ int isqrt_pd(int x)   // floor(sqrt(x)), 0 <= x < 2^30
{
    const float f = (float)max(x, 1);
    int h = __float2int_rz(f * rsqrtf(f));
    h -= (h * h > x);
    h += ((h + 1) * (h + 1) <= x);
    return h;
}
__device__ __forceinline__ int sqi(int v) { return v * v; }

// plan time: F_i and M_i (FP64) over the whole leaf set
__global__ void k_fpd_node(int n, int64_t N, double sigma, double h, const double *__restrict__ delta,
                           const double *__restrict__ c, const int *__restrict__ thr4,
                           double *__restrict__ F, double *__restrict__ M, int K, FpdPoly pc,
                           double *__restrict__ IR2)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int ix = (int)(i % n), iy = (int)(i / n);
    const int X = 2 * ix + 1, Y = 2 * iy + 1;
    const int T4 = thr4[i];
    const double ci = c ? c[i] : 1.0;
    double mxx = 0.0, mxy = 0.0, myy = 0.0;
    const double Ri = delta[i] * n;
    const double ir2 = 1.0 / (Ri * Ri);
    const int r0 = isqrt_pd(T4);
    const int ylo = -((r0 - Y) >> 1) - 1, yhi = (Y + r0) >> 1;       // rows meeting the ball
    for (int ky = ylo; ky <= yhi; ++ky) {
        const int y0 = 2 * ky - Y, y1 = y0 + 2;
        const int e = y0 > 0 ? sqi(y0) : (y1 < 0 ? sqi(y1) : 0);
        if (e > T4) continue;
        const int r = isqrt_pd(T4 - e);
        const int ka = -((r - X) >> 1) - 1, kb = (X + r) >> 1;
        const int dy = ky - iy;
        const bool row_in = ky >= 0 && ky < n;
        for (int kx = ka; kx <= kb; ++kx) {
            const int dx = kx - ix;
            if (dx == 0 && dy == 0) continue;
            const bool in = row_in && kx >= 0 && kx < n;
            double pw = 1.0;                        // p(|o| / R_i), o in cells, R_i = delta_i n
            if (K > 0) {
                const double s2 = (double)(dx * dx + dy * dy) * ir2;
                double t = pc.p[K];
                for (int m = K - 1; m >= 0; --m) t = t * s2 + pc.p[m];
                pw = t;
            }
            const double w = pw * (ci + (in ? (c ? c[(int64_t)ky * n + kx] : 1.0) : ci));
            mxx += w * dx * dx;
            mxy += w * dx * dy;
            myy += w * dy * dy;
        }
    }
    const double di = delta[i];
    F[i] = sigma * h * h * h * h / (2.0 * di * di * di);
    if (IR2) IR2[i] = ir2;
    M[3 * i] = mxx; M[3 * i + 1] = mxy; M[3 * i + 2] = myy;
}

// per-block bounds of |u_x|, |u_y|, |c u_x|, |c u_y| (FP32 products), enlarged by 2^-20
__global__ void __launch_bounds__(256) k_fpd_absmax(int64_t N, const float *__restrict__ ux,
                                                    const float *__restrict__ uy,
                                                    const float *__restrict__ c,
                                                    float *__restrict__ part)
{
    __shared__ float s_w[FPD_FIELDS][8];
    float m[FPD_FIELDS] = { 0.f, 0.f, 0.f, 0.f };
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float a = ux[i], b = uy[i], cc = c[i];
        m[0] = fmaxf(m[0], fabsf(a));
        m[1] = fmaxf(m[1], fabsf(b));
        m[2] = fmaxf(m[2], fabsf(cc * a));
        m[3] = fmaxf(m[3], fabsf(cc * b));
    }
#pragma unroll
    for (int f = 0; f < FPD_FIELDS; ++f) {
        for (int o = 16; o > 0; o >>= 1) m[f] = fmaxf(m[f], __shfl_xor_sync(0xffffffffu, m[f], o));
        if ((threadIdx.x & 31) == 0) s_w[f][threadIdx.x >> 5] = m[f];
    }
    __syncthreads();
    if (threadIdx.x < FPD_FIELDS) {
        float v = 0.f;
        for (int w = 0; w < 8; ++w) v = fmaxf(v, s_w[threadIdx.x][w]);
        part[threadIdx.x * FPD_PARTS + blockIdx.x] = v * (1.f + 0x1p-20f);
    }
}

// scale exponent of a field: q = round(v 2^S) with 2^bits max|q| <= 2^61, where
// 2^bits >= n^2 (2R + 3)^2 (see the header)
__device__ __forceinline__ int fpd_shift(float m, int bits)
{
    if (!(m > 0.f)) return 61 - bits;
    int e1;
    frexpf(m, &e1);                      // m < 2^e1
    return 61 - bits - e1;
}

struct FpdScanArgs {
    int n, bits, nparts;
    const float *ux, *uy, *c, *part;
    int *shifts;                         // [4], written by block 0
    long long *P;                        // [FPD_ARRAYS][N]
    int64_t N;
};

// one warp per row: the ten prefix arrays of the row (quantise, multiply by k and k^2, scan
// with wrapping 64-bit sums); the ten scans advance together, one shuffle each per step
__global__ void __launch_bounds__(128) k_fpd_scan(FpdScanArgs a)
{
    __shared__ int s_sh[FPD_FIELDS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {
        for (int f = 0; f < FPD_FIELDS; ++f) {
            float m = 0.f;
            for (int k = lane; k < a.nparts; k += 32) m = fmaxf(m, a.part[f * FPD_PARTS + k]);
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) s_sh[f] = fpd_shift(m, a.bits);
        }
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x < FPD_FIELDS) a.shifts[threadIdx.x] = s_sh[threadIdx.x];
    const int n = a.n;
    const int row = blockIdx.x * (blockDim.x >> 5) + warp;
    if (row >= n) return;
    const int64_t base = (int64_t)row * n;
    unsigned long long carry[FPD_ARRAYS];
#pragma unroll
    for (int t = 0; t < FPD_ARRAYS; ++t) carry[t] = 0ull;
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int k = k0 + lane;
        unsigned long long v[FPD_ARRAYS];
        if (k < n) {
            const float x = a.ux[base + k], y = a.uy[base + k], cc = a.c[base + k];
            const long long qx = __float2ll_rn(ldexpf(x, s_sh[0]));
            const long long qy = __float2ll_rn(ldexpf(y, s_sh[1]));
            const long long qcx = __float2ll_rn(ldexpf(cc * x, s_sh[2]));
            const long long qcy = __float2ll_rn(ldexpf(cc * y, s_sh[3]));
            const long long kk = k;
            v[0] = (unsigned long long)qx;  v[1] = (unsigned long long)(kk * qx);
            v[2] = (unsigned long long)(kk * kk * qx);
            v[3] = (unsigned long long)qy;  v[4] = (unsigned long long)(kk * qy);
            v[5] = (unsigned long long)qcx; v[6] = (unsigned long long)(kk * qcx);
            v[7] = (unsigned long long)(kk * kk * qcx);
            v[8] = (unsigned long long)qcy; v[9] = (unsigned long long)(kk * qcy);
        } else {
#pragma unroll
            for (int t = 0; t < FPD_ARRAYS; ++t) v[t] = 0ull;
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long w[FPD_ARRAYS];
#pragma unroll
            for (int t = 0; t < FPD_ARRAYS; ++t) w[t] = __shfl_up_sync(0xffffffffu, v[t], o);
            if (lane >= o) {
#pragma unroll
                for (int t = 0; t < FPD_ARRAYS; ++t) v[t] += w[t];
            }
        }
#pragma unroll
        for (int t = 0; t < FPD_ARRAYS; ++t) {
            v[t] += carry[t];
            if (k < n) a.P[(int64_t)t * a.N + base + k] = (long long)v[t];
            carry[t] = __shfl_sync(0xffffffffu, v[t], 31);
        }
    }
}

struct FpdGatherArgs {
    int n;
    int64_t N;
    const int *thr4;
    const double *c;                     // c_i for the factor c_i A (FP64)
    const double *F, *M;
    const long long *P;                  // [FPD_ARRAYS][N]
    const int *shifts;
};

__device__ __forceinline__ unsigned long long pdiff(const long long *P, int64_t row, int ka,
                                                    int kb)
{
    const unsigned long long hi = (unsigned long long)__ldg(P + row + kb);
    const unsigned long long lo = ka > 0 ? (unsigned long long)__ldg(P + row + ka - 1) : 0ull;
    return hi - lo;                              // the run's sum, modulo 2^64
}

__global__ void __launch_bounds__(256) k_fpd_gather(FpdGatherArgs a, const float *__restrict__ ux,
                                                    const float *__restrict__ uy,
                                                    float *__restrict__ outx,
                                                    float *__restrict__ outy)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int n = a.n;
    const int ix = (int)(i % n), iy = (int)(i / n);
    const int X = 2 * ix + 1;
    const int T4 = a.thr4[i];
    const int64_t N = a.N;
    // per group g (0: u, 1: c u) sums over the rows of the run differences of the x-type
    // field (P0 P1 P2): S0, S1, S2, T0 = sum dy P0, T1 = sum dy P1; of the y-type field
    // (P0 P1): U0 = sum dy P0, U1 = sum dy P1, V0 = sum dy^2 P0.  All wrap modulo 2^64: the
    // combinations below are small (sums of o^2 q over one leaf set) and come out exact.
    typedef unsigned long long u64;
    u64 S0[2] = { 0, 0 }, S1[2] = { 0, 0 }, S2[2] = { 0, 0 }, T0[2] = { 0, 0 };
    u64 T1[2] = { 0, 0 }, U0[2] = { 0, 0 }, U1[2] = { 0, 0 }, V0[2] = { 0, 0 };
    for (int t = 0;; ++t) {
        const int e = t == 0 ? 0 : sqi(2 * t - 1);
        if (e > T4) break;
        const int r = isqrt_pd(T4 - e);
        const int ka = max(0, -((r - X) >> 1) - 1);
        const int kb = min(n - 1, (X + r) >> 1);
        for (int s = 0; s < (t > 0 ? 2 : 1); ++s) {
            const int dy = s ? -t : t;
            const int ky = iy + dy;
            if (ky < 0 || ky >= n) continue;
            const int64_t row = (int64_t)ky * n;
            const u64 udy = (u64)(long long)dy, udy2 = (u64)(long long)(dy * dy);
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const long long *Px = a.P + (int64_t)(5 * g) * N;
                const long long *Py = Px + 3 * N;
                const u64 p0 = pdiff(Px, row, ka, kb), p1 = pdiff(Px + N, row, ka, kb),
                          p2 = pdiff(Px + 2 * N, row, ka, kb);
                S0[g] += p0; S1[g] += p1; S2[g] += p2;
                T0[g] += udy * p0; T1[g] += udy * p1;
                const u64 q0 = pdiff(Py, row, ka, kb), q1 = pdiff(Py + N, row, ka, kb);
                U0[g] += udy * q0; U1[g] += udy * q1; V0[g] += udy2 * q0;
            }
        }
    }
    const u64 kx = (u64)ix;
    double A[2][2];                              // [g][component]
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const int sx = a.shifts[2 * g], sy = a.shifts[2 * g + 1];
        const long long xx = (long long)(S2[g] - 2 * kx * S1[g] + kx * kx * S0[g]);  // o_x^2 f_x
        const long long yx = (long long)(T1[g] - kx * T0[g]);                         // o_x o_y f_x
        const long long xy = (long long)(U1[g] - kx * U0[g]);                         // o_x o_y f_y
        const long long yy = (long long)V0[g];                                        // o_y^2 f_y
        A[g][0] = ldexp((double)xx, -sx) + ldexp((double)xy, -sy);
        A[g][1] = ldexp((double)yx, -sx) + ldexp((double)yy, -sy);
    }
    const double ci = a.c[i];
    const double uxi = (double)ux[i], uyi = (double)uy[i];
    const double *Mi = a.M + 3 * i;
    const double Fi = a.F[i];
    outx[i] = (float)(Fi * (ci * A[0][0] + A[1][0] - (Mi[0] * uxi + Mi[1] * uyi)));
    outy[i] = (float)(Fi * (ci * A[0][1] + A[1][1] - (Mi[1] * uxi + Mi[2] * uyi)));
}

// ---------------------------------------------------------------------------
// Polynomial micromodulus, K = 1, 2: the weight p(|o|/R_i) = sum_m beta_m (o_x^2 + o_y^2)^m,
// beta_m = p_m / R_i^{2m}, expands along a leaf row (o_y fixed) into powers of o_x, so the row
// needs the run sums of o_x^e q for e = 0 .. 2K+2 (x-type fields) and 0 .. 2K+1 (y-type):
// from prefix sums of k^m q (k the column) by differences, centred on the node's column with
// the binomial expansion, all modulo 2^64 (the centred values are small and come out exact).
// Over the rows they are accumulated, times powers of o_y, into the exact integer sums
//   Zxe[m][j] = sum dy^{2(m-j)} C_x(2j+2),  Zyo[m][j] = sum dy^{2(m-j)+1} C_y(2j+1),
//   Zxo[m][j] = sum dy^{2(m-j)+1} C_x(2j+1),  Zye[m][j] = sum dy^{2(m-j)+2} C_y(2j),
// and once per node A_x = sum_m beta_m sum_j binom(m, j) (Zxe + Zyo),
// A_y = sum_m beta_m sum_j binom(m, j) (Zxo + Zye) in FP64.  Array layout per group g
// (0: u, 1: c u): x-type powers 0 .. 2K+2, then y-type powers 0 .. 2K+1 (4K + 5 arrays).
// Scale: 2^bits >= (2R + 3)^2 (R + 2)^{2K+2} bounds every such sum.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_fpd_scan_k(FpdScanArgs a, int K)
{
    __shared__ int s_sh[FPD_FIELDS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {
        for (int f = 0; f < FPD_FIELDS; ++f) {
            float m = 0.f;
            for (int k = lane; k < a.nparts; k += 32) m = fmaxf(m, a.part[f * FPD_PARTS + k]);
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) s_sh[f] = fpd_shift(m, a.bits);
        }
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x < FPD_FIELDS) a.shifts[threadIdx.x] = s_sh[threadIdx.x];
    const int n = a.n;
    const int per_g = 4 * K + 5;                     // arrays per group
    const int64_t item = blockIdx.x * (int64_t)(blockDim.x >> 5) + warp;
    if (item >= (int64_t)n * 2 * per_g) return;
    const int row = (int)(item / (2 * per_g));
    const int arr = (int)(item % (2 * per_g));
    const int g = arr / per_g, r = arr % per_g;
    const bool xf = r < 2 * K + 3;                   // x-type field of the group
    const int pw = xf ? r : r - (2 * K + 3);
    const int f = 2 * g + (xf ? 0 : 1);              // shifts: u_x, u_y, c u_x, c u_y
    const int64_t base = (int64_t)row * n;
    const float *__restrict__ src = xf ? a.ux : a.uy;
    unsigned long long carry = 0ull;
    long long *P = a.P + (int64_t)arr * a.N + base;
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int k = k0 + lane;
        unsigned long long v = 0ull;
        if (k < n) {
            float x = src[base + k];
            if (g) x *= a.c[base + k];
            v = (unsigned long long)__float2ll_rn(ldexpf(x, s_sh[f]));
            for (int e = 0; e < pw; ++e) v *= (unsigned long long)k;        // k^pw q, mod 2^64
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long w = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += w;
        }
        v += carry;
        if (k < n) P[k] = (long long)v;
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
}

template <int K>
__global__ void __launch_bounds__(128) k_fpd_gather_k(FpdGatherArgs a, FpdPoly pc,
                                                      const double *__restrict__ ir2v,
                                                      const float *__restrict__ ux,
                                                      const float *__restrict__ uy,
                                                      float *__restrict__ outx,
                                                      float *__restrict__ outy)
{
    typedef unsigned long long u64;
    constexpr int EX = 2 * K + 3, EY = 2 * K + 2, PG = EX + EY;
    constexpr int NJ = (K + 1) * (K + 2) / 2;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int n = a.n;
    const int ix = (int)(i % n), iy = (int)(i / n);
    const int X = 2 * ix + 1;
    const int T4 = a.thr4[i];
    const int64_t N = a.N;
    const u64 ki = (u64)ix;
    // binomial coefficients C(e, m), e <= 2K + 2
    u64 Z[2][4][NJ];                                  // [g][xe, yo, xo, ye][(m, j)]
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int q = 0; q < NJ; ++q) Z[g][t][q] = 0ull;
    for (int t = 0;; ++t) {
        const int e = t == 0 ? 0 : sqi(2 * t - 1);
        if (e > T4) break;
        const int r = isqrt_pd(T4 - e);
        const int ka = max(0, -((r - X) >> 1) - 1);
        const int kb = min(n - 1, (X + r) >> 1);
        for (int s = 0; s < (t > 0 ? 2 : 1); ++s) {
            const int dy = s ? -t : t;
            const int ky = iy + dy;
            if (ky < 0 || ky >= n) continue;
            const int64_t row = (int64_t)ky * n;
            u64 dyp[EX];                              // dy^a, a <= 2K + 2
            dyp[0] = 1ull;
#pragma unroll
            for (int q = 1; q < EX; ++q) dyp[q] = dyp[q - 1] * (u64)(long long)dy;
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const long long *Pg = a.P + (int64_t)(g * PG) * N;
                u64 D[EX], Cx[EX], Cy[EY];
#pragma unroll
                for (int m = 0; m < EX; ++m) D[m] = pdiff(Pg + (int64_t)m * N, row, ka, kb);
#pragma unroll
                for (int q = 0; q < EX; ++q) {           // centred: sum C(q,m) (-k_i)^{q-m} D_m
                    u64 acc = 0ull, pk = 1ull;
#pragma unroll
                    for (int m = q; m >= 0; --m) {
                        u64 bin = 1ull;
#pragma unroll
                        for (int z = 0; z < q - m; ++z) bin = bin * (u64)(m + 1 + z) / (u64)(1 + z);
                        const u64 term = bin * pk * D[m];
                        acc += ((q - m) & 1) ? (u64)(0ull - term) : term;
                        pk *= ki;
                    }
                    Cx[q] = acc;
                }
#pragma unroll
                for (int m = 0; m < EY; ++m) D[m] = pdiff(Pg + (int64_t)(EX + m) * N, row, ka, kb);
#pragma unroll
                for (int q = 0; q < EY; ++q) {
                    u64 acc = 0ull, pk = 1ull;
#pragma unroll
                    for (int m = q; m >= 0; --m) {
                        u64 bin = 1ull;
#pragma unroll
                        for (int z = 0; z < q - m; ++z) bin = bin * (u64)(m + 1 + z) / (u64)(1 + z);
                        const u64 term = bin * pk * D[m];
                        acc += ((q - m) & 1) ? (u64)(0ull - term) : term;
                        pk *= ki;
                    }
                    Cy[q] = acc;
                }
                int q = 0;
#pragma unroll
                for (int m = 0; m <= K; ++m)
#pragma unroll
                    for (int j = 0; j <= m; ++j, ++q) {
                        Z[g][0][q] += dyp[2 * (m - j)] * Cx[2 * j + 2];
                        Z[g][1][q] += dyp[2 * (m - j) + 1] * Cy[2 * j + 1];
                        Z[g][2][q] += dyp[2 * (m - j) + 1] * Cx[2 * j + 1];
                        Z[g][3][q] += dyp[2 * (m - j) + 2] * Cy[2 * j];
                    }
            }
        }
    }
    const double ir2 = ir2v[i];                     // 1 / R_i^2, R_i = delta_i n
    double A[2][2];
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const int sx = a.shifts[2 * g], sy = a.shifts[2 * g + 1];
        double ax = 0.0, ay = 0.0, beta = 1.0;
        int q = 0;
#pragma unroll
        for (int m = 0; m <= K; ++m) {
            double bx = 0.0, by = 0.0, bin = 1.0;
#pragma unroll
            for (int j = 0; j <= m; ++j, ++q) {
                bx += bin * (ldexp((double)(long long)Z[g][0][q], -sx) +
                             ldexp((double)(long long)Z[g][1][q], -sy));
                by += bin * (ldexp((double)(long long)Z[g][2][q], -sx) +
                             ldexp((double)(long long)Z[g][3][q], -sy));
                bin = bin * (m - j) / (j + 1);
            }
            ax += pc.p[m] * beta * bx;
            ay += pc.p[m] * beta * by;
            beta *= ir2;
        }
        A[g][0] = ax;
        A[g][1] = ay;
    }
    const double ci = a.c[i];
    const double uxi = (double)ux[i], uyi = (double)uy[i];
    const double *Mi = a.M + 3 * i;
    const double Fi = a.F[i];
    outx[i] = (float)(Fi * (ci * A[0][0] + A[1][0] - (Mi[0] * uxi + Mi[1] * uyi)));
    outy[i] = (float)(Fi * (ci * A[0][1] + A[1][1] - (Mi[1] * uxi + Mi[2] * uyi)));
}

// ---------------------------------------------------------------------------
// 3-D, K = 0: xi = o h with o = (o_x, o_y, o_z); along a leaf row (o_y, o_z fixed) the x-type
// field needs the run sums of q, k q, k^2 q and the y- and z-type fields those of q and k q:
//   (o o^T q)_x = o_x^2 q_x + o_x o_y q_y + o_x o_z q_z,
//   (o o^T q)_y = o_x o_y q_x + o_y^2 q_y + o_y o_z q_z,
//   (o o^T q)_z = o_x o_z q_x + o_y o_z q_y + o_z^2 q_z,
// seven prefix arrays per group (u, c u), fourteen in all, with the rows and runs of the
// scalar leaf-row gather in 3-D (vertical gap from the row's y and z gaps).  Sums wrap modulo
// 2^64; 2^bits >= (2R + 3)^3 (R + 2)^2 bounds every per-node combination, which is exact.
// ---------------------------------------------------------------------------
constexpr int FPD3_FIELDS = 6;                  // u_x, u_y, u_z, c u_x, c u_y, c u_z
constexpr int FPD3_ARRAYS = 14;                 // per group: x P0 P1 P2, y P0 P1, z P0 P1

// half-unit gap^2 from a node at 2 i + 1 to cell k (0 for its own cell)
__device__ __forceinline__ int gap2_pd(int k, int I)
{
    const int lo = 2 * k - I, hi = lo + 2;
    return lo > 0 ? lo * lo : (hi < 0 ? hi * hi : 0);
}

// plan time, 3-D: F_i = sigma h^5 / (2 delta_i^3) and the six entries of
// M_i = sum_{k in LS(i)} (c_i + c_k) o o^T (xx, xy, xz, yy, yz, zz; FP64)
__global__ void k_fpd_node3(int n, int64_t N, double sigma, double h,
                            const double *__restrict__ delta, const double *__restrict__ c,
                            const int *__restrict__ thr4, double *__restrict__ F,
                            double *__restrict__ M)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((int64_t)n * n));
    const int X = 2 * ix + 1, Y = 2 * iy + 1, Z = 2 * iz + 1;
    const int T4 = thr4[i];
    const double ci = c ? c[i] : 1.0;
    const int r0 = isqrt_pd(T4);
    double m[6] = { 0, 0, 0, 0, 0, 0 };
    const int zlo = -((r0 - Z) >> 1) - 1, zhi = (Z + r0) >> 1;
    const int ylo = -((r0 - Y) >> 1) - 1, yhi = (Y + r0) >> 1;
    for (int kz = zlo; kz <= zhi; ++kz) {
        const int ez = gap2_pd(kz, Z);
        if (ez > T4) continue;
        for (int ky = ylo; ky <= yhi; ++ky) {
            const int e = ez + gap2_pd(ky, Y);
            if (e > T4) continue;
            const int r = isqrt_pd(T4 - e);
            const int ka = -((r - X) >> 1) - 1, kb = (X + r) >> 1;
            const int dy = ky - iy, dz = kz - iz;
            const bool row_in = ky >= 0 && ky < n && kz >= 0 && kz < n;
            for (int kx = ka; kx <= kb; ++kx) {
                const int dx = kx - ix;
                if (dx == 0 && dy == 0 && dz == 0) continue;
                const bool in = row_in && kx >= 0 && kx < n;
                const double w =
                    ci + (in ? (c ? c[((int64_t)kz * n + ky) * n + kx] : 1.0) : ci);
                m[0] += w * dx * dx; m[1] += w * dx * dy; m[2] += w * dx * dz;
                m[3] += w * dy * dy; m[4] += w * dy * dz; m[5] += w * dz * dz;
            }
        }
    }
    const double di = delta[i];
    F[i] = sigma * h * h * h * h * h / (2.0 * di * di * di);
#pragma unroll
    for (int t = 0; t < 6; ++t) M[6 * i + t] = m[t];
}

// per-block bounds of the six fields (FP32 products), enlarged by 2^-20
__global__ void __launch_bounds__(256) k_fpd_absmax3(int64_t N, const float *__restrict__ u,
                                                     const float *__restrict__ c,
                                                     float *__restrict__ part)
{
    __shared__ float s_w[FPD3_FIELDS][8];
    float m[FPD3_FIELDS] = { 0.f, 0.f, 0.f, 0.f, 0.f, 0.f };
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float cc = c[i];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const float v = u[(int64_t)f * N + i];
            m[f] = fmaxf(m[f], fabsf(v));
            m[3 + f] = fmaxf(m[3 + f], fabsf(cc * v));
        }
    }
#pragma unroll
    for (int f = 0; f < FPD3_FIELDS; ++f) {
        for (int o = 16; o > 0; o >>= 1) m[f] = fmaxf(m[f], __shfl_xor_sync(0xffffffffu, m[f], o));
        if ((threadIdx.x & 31) == 0) s_w[f][threadIdx.x >> 5] = m[f];
    }
    __syncthreads();
    if (threadIdx.x < FPD3_FIELDS) {
        float v = 0.f;
        for (int w = 0; w < 8; ++w) v = fmaxf(v, s_w[threadIdx.x][w]);
        part[threadIdx.x * FPD_PARTS + blockIdx.x] = v * (1.f + 0x1p-20f);
    }
}

struct Fpd3ScanArgs {
    int n, bits, nparts;
    const float *u, *c, *part;          // u: [3][N]
    int *shifts;                        // [6], written by block 0
    long long *P;                       // [14][N]
    int64_t N;
};

// one warp per leaf row (n^2 rows): the fourteen prefix arrays of the row, each field rounded
// once to a multiple of 2^-S (its own S), times k and k^2 modulo 2^64, scanned with shuffles
__global__ void __launch_bounds__(128) k_fpd_scan3(Fpd3ScanArgs a)
{
    __shared__ int s_sh[FPD3_FIELDS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {
        for (int f = 0; f < FPD3_FIELDS; ++f) {
            float m = 0.f;
            for (int k = lane; k < a.nparts; k += 32) m = fmaxf(m, a.part[f * FPD_PARTS + k]);
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) s_sh[f] = fpd_shift(m, a.bits);
        }
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x < FPD3_FIELDS) a.shifts[threadIdx.x] = s_sh[threadIdx.x];
    const int n = a.n;
    const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + warp;
    if (row >= (int64_t)n * n) return;
    const int64_t base = row * n, N = a.N;
    typedef unsigned long long u64;
    u64 carry[FPD3_ARRAYS];
#pragma unroll
    for (int t = 0; t < FPD3_ARRAYS; ++t) carry[t] = 0ull;
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int k = k0 + lane;
        u64 v[FPD3_ARRAYS];
        if (k < n) {
            const float cc = a.c[base + k];
            const u64 kk = (u64)k;
#pragma unroll
            for (int g = 0; g < 2; ++g) {
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    float x = a.u[(int64_t)f * N + base + k];
                    if (g) x *= cc;
                    const u64 q = (u64)__float2ll_rn(ldexpf(x, s_sh[3 * g + f]));
                    const int t0 = 7 * g + (f == 0 ? 0 : (f == 1 ? 3 : 5));
                    v[t0] = q;
                    v[t0 + 1] = kk * q;
                    if (f == 0) v[t0 + 2] = kk * kk * q;
                }
            }
        } else {
#pragma unroll
            for (int t = 0; t < FPD3_ARRAYS; ++t) v[t] = 0ull;
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int t = 0; t < FPD3_ARRAYS; ++t) {
                const u64 w = __shfl_up_sync(0xffffffffu, v[t], o);
                if (lane >= o) v[t] += w;
            }
        }
#pragma unroll
        for (int t = 0; t < FPD3_ARRAYS; ++t) {
            v[t] += carry[t];
            if (k < n) a.P[(int64_t)t * N + base + k] = (long long)v[t];
            carry[t] = __shfl_sync(0xffffffffu, v[t], 31);
        }
    }
}

// per node: over the leaf rows (dy, dz) of its ball, the run differences of the fourteen
// arrays, accumulated (times dy, dz, dy^2, dy dz, dz^2) into exact sums modulo 2^64, then
// centred on the node's column and combined in FP64 with each field's scale
__global__ void __launch_bounds__(128) k_fpd_gather3(FpdGatherArgs a, const float *__restrict__ u,
                                                     float *__restrict__ out)
{
    typedef unsigned long long u64;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int n = a.n;
    const int64_t N = a.N;
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((int64_t)n * n));
    const int X = 2 * ix + 1;
    const int T4 = a.thr4[i];
    // per group: SX0 SX1 SX2, TY0 TY1 (dy x), TZ0 TZ1 (dz x), UY0 UY1 (dy y), VYY (dy^2 y0),
    // VYZY (dy dz y0), WZ0 WZ1 (dz z), VZZ (dz^2 z0), VYZZ (dy dz z0)
    u64 acc[2][15];
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
        for (int t = 0; t < 15; ++t) acc[g][t] = 0ull;
    for (int tz = 0;; ++tz) {
        const int ez = tz == 0 ? 0 : sqi(2 * tz - 1);
        if (ez > T4) break;
        for (int ty = 0;; ++ty) {
            const int e = ez + (ty == 0 ? 0 : sqi(2 * ty - 1));
            if (e > T4) break;
            const int r = isqrt_pd(T4 - e);
            const int ka = max(0, -((r - X) >> 1) - 1);
            const int kb = min(n - 1, (X + r) >> 1);
            for (int sz = 0; sz < (tz > 0 ? 2 : 1); ++sz) {
                const int dz = sz ? -tz : tz;
                const int kz = iz + dz;
                if (kz < 0 || kz >= n) continue;
                for (int sy = 0; sy < (ty > 0 ? 2 : 1); ++sy) {
                    const int dy = sy ? -ty : ty;
                    const int ky = iy + dy;
                    if (ky < 0 || ky >= n) continue;
                    const int64_t row = ((int64_t)kz * n + ky) * n;
                    const u64 uy = (u64)(long long)dy, uz = (u64)(long long)dz;
                    const u64 uyy = uy * uy, uyz = uy * uz, uzz = uz * uz;
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
                        const long long *Pg = a.P + (int64_t)(7 * g) * N;
                        const u64 x0 = pdiff(Pg, row, ka, kb), x1 = pdiff(Pg + N, row, ka, kb),
                                  x2 = pdiff(Pg + 2 * N, row, ka, kb);
                        const u64 y0 = pdiff(Pg + 3 * N, row, ka, kb),
                                  y1 = pdiff(Pg + 4 * N, row, ka, kb);
                        const u64 z0 = pdiff(Pg + 5 * N, row, ka, kb),
                                  z1 = pdiff(Pg + 6 * N, row, ka, kb);
                        u64 *A = acc[g];
                        A[0] += x0; A[1] += x1; A[2] += x2;
                        A[3] += uy * x0; A[4] += uy * x1;
                        A[5] += uz * x0; A[6] += uz * x1;
                        A[7] += uy * y0; A[8] += uy * y1;
                        A[9] += uyy * y0; A[10] += uyz * y0;
                        A[11] += uz * z0; A[12] += uz * z1;
                        A[13] += uzz * z0; A[14] += uyz * z0;
                    }
                }
            }
        }
    }
    const u64 kx = (u64)ix;
    double R[2][3];                              // [g][component]
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const u64 *A = acc[g];
        const int sx = a.shifts[3 * g], sy = a.shifts[3 * g + 1], sz = a.shifts[3 * g + 2];
        const long long xx = (long long)(A[2] - 2 * kx * A[1] + kx * kx * A[0]);   // o_x^2 q_x
        const long long yx = (long long)(A[4] - kx * A[3]);                        // o_x o_y q_x
        const long long zx = (long long)(A[6] - kx * A[5]);                        // o_x o_z q_x
        const long long xy = (long long)(A[8] - kx * A[7]);                        // o_x o_y q_y
        const long long yy = (long long)A[9];                                      // o_y^2 q_y
        const long long zy = (long long)A[10];                                     // o_y o_z q_y
        const long long xz = (long long)(A[12] - kx * A[11]);                      // o_x o_z q_z
        const long long zz = (long long)A[13];                                     // o_z^2 q_z
        const long long yz = (long long)A[14];                                     // o_y o_z q_z
        R[g][0] = ldexp((double)xx, -sx) + ldexp((double)xy, -sy) + ldexp((double)xz, -sz);
        R[g][1] = ldexp((double)yx, -sx) + ldexp((double)yy, -sy) + ldexp((double)yz, -sz);
        R[g][2] = ldexp((double)zx, -sx) + ldexp((double)zy, -sy) + ldexp((double)zz, -sz);
    }
    const double ci = a.c[i];
    const double u0 = (double)u[i], u1 = (double)u[N + i], u2 = (double)u[2 * N + i];
    const double *Mi = a.M + 6 * i;
    const double Fi = a.F[i];
    out[i] = (float)(Fi * (ci * R[0][0] + R[1][0] - (Mi[0] * u0 + Mi[1] * u1 + Mi[2] * u2)));
    out[N + i] = (float)(Fi * (ci * R[0][1] + R[1][1] - (Mi[1] * u0 + Mi[3] * u1 + Mi[4] * u2)));
    out[2 * N + i] = (float)(Fi * (ci * R[0][2] + R[1][2] - (Mi[2] * u0 + Mi[4] * u1 + Mi[5] * u2)));
}

}  // namespace

// plan-time set-up, 3-D (K = 0, n = 2^L <= 256): F, M (six per node), the fourteen prefix
// arrays (112 bytes per node) and the bounds workspace
static nl_status fast_pd3_plan_init(nl_plan *p, const double *delta_dev, const double *c_dev,
                                    cudaStream_t st)
{
    if (p->L < 0 || p->n > 256 || !p->thr4 || p->K != 0) return NL_OK;
    const double rr = 2.0 * p->Rmax + 3;
    const double bound = rr * rr * rr * (p->Rmax + 2.0) * (p->Rmax + 2.0);
    if (bound > 0x1p48) return NL_OK;
    const int64_t N = p->N;
    auto alloc = [&](void **ptr, size_t bytes) -> nl_status {
        if (cudaMalloc(ptr, bytes ? bytes : 1) != cudaSuccess) {
            nl_set_error("cudaMalloc(%zu) for the fast peridynamic path failed", bytes);
            return NL_ENOMEM;
        }
        p->device_bytes += bytes;
        return NL_OK;
    };
    nl_status s;
    if ((s = alloc((void **)&p->fpd_F, N * sizeof(double))) != NL_OK) return s;
    if ((s = alloc((void **)&p->fpd_M, 6 * N * sizeof(double))) != NL_OK) return s;
    if ((s = alloc((void **)&p->fpd_P, (size_t)FPD3_ARRAYS * N * sizeof(long long))) != NL_OK)
        return s;
    if ((s = alloc((void **)&p->fpd_aux, FPD3_FIELDS * FPD_PARTS * sizeof(float) + 64)) != NL_OK)
        return s;
    p->fpd_bits = (int)std::ceil(std::log2(bound));
    k_fpd_node3<<<(unsigned)((N + 127) / 128), 128, 0, st>>>(p->n, N, p->sigma, p->h, delta_dev,
                                                            c_dev, p->thr4, p->fpd_F, p->fpd_M);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

// plan-time set-up (2-D NL_PD_BOND plans with n = 2^L <= 8192)
nl_status nl_fast_pd_plan_init(nl_plan *p, const double *delta_dev, const double *c_dev,
                               cudaStream_t st)
{
    if (p->d == 3) return fast_pd3_plan_init(p, delta_dev, c_dev, st);
    if (p->d != 2 || p->L < 0 || p->n > 8192 || !p->thr4 || p->K > 2) return NL_OK;
    // 2^bits bounds every per-node integer sum: n^2 (2 Rmax + 3)^2 for K = 0, (2 Rmax + 3)^2
    // (Rmax + 2)^{2K+2} for K >= 1; at least 2^13 levels must remain for max|v|
    const double rr = 2.0 * p->Rmax + 3;
    const double bound = p->K == 0 ? (double)p->n * p->n * rr * rr
                                   : rr * rr * std::pow(p->Rmax + 2.0, 2.0 * p->K + 2.0);
    if (bound > 0x1p48) return NL_OK;
    const int64_t N = p->N;
    auto alloc = [&](void **ptr, size_t bytes) -> nl_status {
        if (cudaMalloc(ptr, bytes ? bytes : 1) != cudaSuccess) {
            nl_set_error("cudaMalloc(%zu) for the fast peridynamic path failed", bytes);
            return NL_ENOMEM;
        }
        p->device_bytes += bytes;
        return NL_OK;
    };
    nl_status s;
    if ((s = alloc((void **)&p->fpd_F, N * sizeof(double))) != NL_OK) return s;
    if ((s = alloc((void **)&p->fpd_M, 3 * N * sizeof(double))) != NL_OK) return s;
    if (p->K > 0 && (s = alloc((void **)&p->fpd_ir2, N * sizeof(double))) != NL_OK) return s;
    const int arrays = p->K == 0 ? FPD_ARRAYS : 8 * p->K + 10;
    if ((s = alloc((void **)&p->fpd_P, (size_t)arrays * N * sizeof(long long))) != NL_OK) return s;
    if ((s = alloc((void **)&p->fpd_aux, FPD_FIELDS * FPD_PARTS * sizeof(float) + 64)) != NL_OK) return s;
    p->fpd_bits = (int)std::ceil(std::log2(bound));
    FpdPoly pc;
    for (int m = 0; m < 8; ++m) pc.p[m] = p->poly[m];
    k_fpd_node<<<(unsigned)((N + 127) / 128), 128, 0, st>>>(p->n, N, p->sigma, p->h, delta_dev,
                                                           c_dev, p->thr4, p->fpd_F, p->fpd_M,
                                                           p->K, pc, p->fpd_ir2);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

// one FP32 right-hand side: bounds, the ten prefix arrays, the gather
nl_status nl_fast_pd_launch(nl_plan *p, const float *u, float *Lu, int nrhs, cudaStream_t st)
{
    if (!p->fpd_P) {
        nl_set_error("nl_apply_fast: the fast peridynamic path needs n = 2^L and a horizon "
                     "whose integer sums fit 64 bits, with n <= 8192 and K <= 2 in 2-D, "
                     "n <= 256 and K = 0 in 3-D");
        return NL_EUNSUPPORTED;
    }
    const int64_t N = p->N;
    if (p->d == 3) {
        float *part = (float *)p->fpd_aux;
        int *shifts = (int *)((unsigned char *)p->fpd_aux + FPD3_FIELDS * FPD_PARTS * sizeof(float));
        int64_t per = (N + FPD_PARTS - 1) / FPD_PARTS;
        if (per < 2048) per = 2048;
        const int nparts = (int)((N + per - 1) / per);
        for (int r = 0; r < nrhs; ++r) {
            const float *ur = u + (int64_t)r * 3 * N;
            float *lr = Lu + (int64_t)r * 3 * N;
            k_fpd_absmax3<<<nparts, 256, 0, st>>>(N, ur, p->b32, part);
            Fpd3ScanArgs sa;
            sa.n = p->n; sa.bits = p->fpd_bits; sa.nparts = nparts;
            sa.u = ur; sa.c = p->b32; sa.part = part; sa.shifts = shifts;
            sa.P = p->fpd_P; sa.N = N;
            const int64_t rows = (int64_t)p->n * p->n;
            k_fpd_scan3<<<(unsigned)((rows + 3) / 4), 128, 0, st>>>(sa);
            FpdGatherArgs ga;
            ga.n = p->n; ga.N = N; ga.thr4 = p->thr4; ga.c = p->b64;
            ga.F = p->fpd_F; ga.M = p->fpd_M; ga.P = p->fpd_P; ga.shifts = shifts;
            k_fpd_gather3<<<(unsigned)((N + 127) / 128), 128, 0, st>>>(ga, ur, lr);
            NL_CUDA_TRY(cudaGetLastError());
        }
        return NL_OK;
    }
    float *part = (float *)p->fpd_aux;
    int *shifts = (int *)((unsigned char *)p->fpd_aux + FPD_FIELDS * FPD_PARTS * sizeof(float));
    int64_t per = (N + FPD_PARTS - 1) / FPD_PARTS;
    if (per < 2048) per = 2048;
    const int nparts = (int)((N + per - 1) / per);
    for (int r = 0; r < nrhs; ++r) {
        const float *ux = u + (int64_t)r * 2 * N, *uy = ux + N;
        float *ox = Lu + (int64_t)r * 2 * N, *oy = ox + N;
        k_fpd_absmax<<<nparts, 256, 0, st>>>(N, ux, uy, p->b32, part);
        FpdScanArgs sa;
        sa.n = p->n; sa.bits = p->fpd_bits; sa.nparts = nparts;
        sa.ux = ux; sa.uy = uy; sa.c = p->b32; sa.part = part; sa.shifts = shifts;
        sa.P = p->fpd_P; sa.N = N;
        FpdGatherArgs ga;
        ga.n = p->n; ga.N = N; ga.thr4 = p->thr4; ga.c = p->b64;
        ga.F = p->fpd_F; ga.M = p->fpd_M; ga.P = p->fpd_P; ga.shifts = shifts;
        if (p->K == 0) {
            k_fpd_scan<<<(unsigned)((p->n + 3) / 4), 128, 0, st>>>(sa);
            k_fpd_gather<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(ga, ux, uy, ox, oy);
        } else {
            const int64_t items = (int64_t)p->n * 2 * (4 * p->K + 5);
            k_fpd_scan_k<<<(unsigned)((items + 3) / 4), 128, 0, st>>>(sa, p->K);
            FpdPoly pc;
            for (int m = 0; m < 8; ++m) pc.p[m] = p->poly[m];
            const unsigned gg = (unsigned)((N + 127) / 128);
            if (p->K == 1) k_fpd_gather_k<1><<<gg, 128, 0, st>>>(ga, pc, p->fpd_ir2, ux, uy, ox, oy);
            else k_fpd_gather_k<2><<<gg, 128, 0, st>>>(ga, pc, p->fpd_ir2, ux, uy, ox, oy);
        }
        NL_CUDA_TRY(cudaGetLastError());
    }
    return NL_OK;
}
