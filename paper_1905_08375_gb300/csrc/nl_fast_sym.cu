// nl_fast_sym.cu -- the fast path for the symmetrised (divergence-type) polynomial operator,
// K = 0 here and K = 1..3 below (a project extension of Sec. 3, which treats the one-sided
// C(x) delta(x) form only;
// the symmetric pairing w_ij + w_ji is the divergence type of Sec. 2 case (b)):
//
//   (L u)_i = sigma h^d sum_k (w_i(k) + w_k(i))/2 a_i a_k (u_k - u_i),
//   w_i(k)  = [cell k meets the open ball of node i] delta_i^{-(d+2)}   (p = 1),
//
// k over every lattice cell, with u_k = 0, a_k = a_i and delta_k = delta_i outside Omega.  The
// first half is the one-sided leaf-set operator of nl_apply_fast (discrete self term).  The
// second half, with c_k = a_k delta_k^{-(d+2)}, is
//
//   half2_i = sigma h^d a_i [ S_i - u_i T_i ],  S_i = sum_{k in Omega, i in LS(k)} c_k u_k,
//                                               T_i = sum_{k, i in LS(k)} c_k   (plan time),
//
// the transpose of the leaf-row gather: each node k adds v_k = c_k u_k at the first cell of
// every leaf row of its own leaf set (inside Omega) and -v_k one past the last, and one prefix
// sum per row turns those difference arrays into S.  FP32 data: v_k rounded once to a multiple
// of 2^-S (N max|c u| 2^S < 2^62), so the atomics add exact integers and the order of the
// scatters cannot change the result; FP64 data: FP64 atomics.  The result is
//   L u = (half1 + half2) / 2.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "nl_internal.cuh"

namespace {

__device__ __forceinline__ int sym_sq(int v) { return v * v; }

// floor(sqrt(x)) for 0 <= x < 2^30 (approximate reciprocal square root, then exact
// integer corrections)
__device__ __forceinline__ int sym_isqrt(int x)
{
    const float f = (float)max(x, 1);
    int h = __float2int_rz(f * rsqrtf(f));
    h -= (h * h > x);
    h += ((h + 1) * (h + 1) <= x);
    return h;
}

struct SymArgs {
    int d, n, coef, K;
    int64_t N;
    double sigma, hd;
    double p[8];                      // p_0 .. p_K of p^{2K} (p(s) = sum_m p_m s^{2m})
    const int *thr4;
    double *ir2;                      // K >= 1: 1 / R_k^2, R_k = delta_k n
    const double *delta, *acoef;      // plan time only (device copies)
    double *c64;                      // c_k = a_k delta_k^{-(d+2)}
    float *c32;
    double *T;                        // sum over k with i in LS(k) of c_k
    double *G64;                      // sigma h^d a_i
    float *G32;
    double *diag;                     // -L_ii (Jacobi)
    const double *fastF, *selfS;      // the one-sided operator's factor and self term
};

// Plan time, per node i: c_i = a_i delta_i^{-(d+2)} and G_i = sigma h^d a_i.
__global__ void k_sym_coef(SymArgs a)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const double ai = a.coef == NL_COEF_XY ? a.acoef[i] : 1.0;
    const double ci = ai * pow(a.delta[i], -(a.d + 2.0));
    a.c64[i] = ci;
    a.c32[i] = (float)ci;
    const double Gi = a.sigma * a.hd * ai;
    a.G64[i] = Gi;
    a.G32[i] = (float)Gi;
    if (a.ir2) {
        const double R = a.delta[i] * a.n;
        a.ir2[i] = 1.0 / (R * R);
    }
}

// p(|o|^2 / R^2) = sum_m p_m (|o|^2 ir2)^m (Horner)
__device__ __forceinline__ double sym_poly(const SymArgs &a, int o2, double ir2)
{
    const double t = (double)o2 * ir2;
    double w = a.p[a.K];
    for (int m = a.K - 1; m >= 0; --m) w = w * t + a.p[m];
    return w;
}

// Plan time, per node i: T_i by the definition -- every cell k of the box of radius B around i
// whose own leaf set reaches i (the half-unit gap from node k to cell i, per axis 2|o| - 1, 0
// for o = 0, squared and summed, at most thr4_k; cells outside Omega take the node's own
// horizon and coefficient, so there the test is the node's own), each with its weight
// c_k p(|o|^2 / R_k^2) (p = 1 for K = 0) -- and the Jacobi diagonal
//   -L_ii = [fastF_i (selfS_i - h^d p_0 b_i) + G_i (T_i - p_0 c_i)] / 2.
__global__ void k_sym_node(SymArgs a, int B)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int n = a.n, d = a.d;
    const int ix = (int)(i % n);
    const int iy = d > 1 ? (int)((i / n) % n) : 0;
    const int iz = d > 2 ? (int)(i / ((int64_t)n * n)) : 0;
    const double ci = a.c64[i];
    const int T4i = a.thr4[i];
    const int bz = d > 2 ? B : 0, by = d > 1 ? B : 0;
    double T = 0.0;
    for (int oz = -bz; oz <= bz; ++oz) {
        const int gz = oz ? 2 * abs(oz) - 1 : 0;
        const int kz = iz + oz;
        const bool inz = d < 3 || (kz >= 0 && kz < n);
        for (int oy = -by; oy <= by; ++oy) {
            const int gy = oy ? 2 * abs(oy) - 1 : 0;
            const int ky = iy + oy;
            const bool iny = inz && (d < 2 || (ky >= 0 && ky < n));
            const int eyz = gy * gy + gz * gz;
            const int oyz = oy * oy + oz * oz;
            for (int ox = -B; ox <= B; ++ox) {
                const int gx = ox ? 2 * abs(ox) - 1 : 0;
                const int e = gx * gx + eyz;
                const int kx = ix + ox;
                if (iny && kx >= 0 && kx < n) {
                    const int64_t k = kx + (int64_t)n * (ky + (int64_t)n * kz);
                    if (e <= a.thr4[k])
                        T += a.K ? a.c64[k] * sym_poly(a, ox * ox + oyz, a.ir2[k]) : a.c64[k];
                } else if (e <= T4i) {
                    T += a.K ? ci * sym_poly(a, ox * ox + oyz, a.ir2[i]) : ci;
                }
            }
        }
    }
    const double ai = a.coef == NL_COEF_XY ? a.acoef[i] : 1.0;
    a.T[i] = T;
    const double p0 = a.K ? a.p[0] : 1.0;
    a.diag[i] = 0.5 * (a.fastF[i] * (a.selfS[i] - a.hd * p0 * ai) + a.G64[i] * (T - p0 * ci));
}

// scale exponent from the per-block bounds of |c u| (the arithmetic of the one-sided route)
__device__ __forceinline__ int sym_block_shift(const float *part, int nparts, int64_t N,
                                               unsigned int *mx_out)
{
    __shared__ float s_w[32];
    __shared__ int s_sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    float m = 0.f;
    for (int k = tid; k < nparts; k += blockDim.x) m = fmaxf(m, part[k]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) s_w[warp] = m;
    __syncthreads();
    if (tid == 0) {
        float mm = 0.f;
        for (int w = 0; w < nw; ++w) mm = fmaxf(mm, s_w[w]);
        if (blockIdx.x == 0 && mx_out) *mx_out = __float_as_uint(mm);
        int sh = 62;
        if (mm > 0.f) {
            int e1, e2;
            frexpf(mm, &e1);
            frexpf((float)N, &e2);
            sh = 62 - e1 - e2;
        }
        s_sh = sh;
    }
    __syncthreads();
    return s_sh;
}

__device__ __forceinline__ int sym_shift_of(int64_t N, const unsigned int *mx)
{
    const float m = __uint_as_float(*mx);
    if (!(m > 0.f)) return 62;
    int e1, e2;
    frexpf(m, &e1);
    frexpf((float)N, &e2);
    return 62 - e1 - e2;
}

template <typename Acc>
__device__ __forceinline__ void sym_add(Acc *p, Acc v)
{
    if constexpr (sizeof(Acc) == 8 && !std::is_floating_point<Acc>::value)
        atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
    else
        atomicAdd(p, v);
}

// the leaf rows of node k's leaf set: rows (and slabs) at gap index t (half-unit gap 2t - 1,
// 0 for the node's own row) carry the run of cells whose x-gap^2 fits in the rest of thr4_k;
// +v at the run's first cell inside Omega, -v one past its last (when that is inside Omega)
template <typename Acc>
__device__ __forceinline__ void sym_row(Acc *D, int64_t rowoff, int n, int X, int r, Acc v)
{
    const int ka = max(0, -((r - X) >> 1) - 1);
    const int kb = min(n - 1, (X + r) >> 1);
    sym_add(D + rowoff + ka, v);
    if (kb + 1 < n) sym_add(D + rowoff + kb + 1, (Acc)(-v));
}

template <int DIM, typename T, typename Acc>
__global__ void __launch_bounds__(256) k_sym_scatter(SymArgs a, const T *__restrict__ u,
                                                     Acc *__restrict__ D,
                                                     const float *__restrict__ part, int nparts,
                                                     unsigned int *mx)
{
    int sh = 0;
    if constexpr (!std::is_floating_point<Acc>::value) sh = sym_block_shift(part, nparts, a.N, mx);
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= a.N) return;
    const int n = a.n;
    const int kx = (int)(k % n);
    const int ky = DIM > 1 ? (int)((k / n) % n) : 0;
    const int kz = DIM > 2 ? (int)(k / ((int64_t)n * n)) : 0;
    Acc v;
    if constexpr (std::is_floating_point<Acc>::value) v = (Acc)(a.c64[k] * (double)u[k]);
    else v = (Acc)__float2ll_rn(ldexpf(a.c32[k] * (float)u[k], sh));
    if (v == (Acc)0) return;
    const int X = 2 * kx + 1;
    const int T4 = a.thr4[k];
    if (DIM == 1) {
        sym_row<Acc>(D, 0, n, X, sym_isqrt(T4), v);
        return;
    }
    const int64_t pl = (int64_t)n * n;
    for (int tz = 0; tz <= (DIM > 2 ? n : 0); ++tz) {
        const int ez = tz == 0 ? 0 : sym_sq(2 * tz - 1);
        if (ez > T4) break;
        for (int sz = 0; sz < (DIM > 2 && tz > 0 ? 2 : 1); ++sz) {
            const int z = DIM > 2 ? (sz ? kz - tz : kz + tz) : 0;
            if (z < 0 || z >= (DIM > 2 ? n : 1)) continue;
            for (int ty = 0;; ++ty) {
                const int e = ez + (ty == 0 ? 0 : sym_sq(2 * ty - 1));
                if (e > T4) break;
                const int r = sym_isqrt(T4 - e);
                if (ky + ty < n) sym_row<Acc>(D, pl * z + (int64_t)n * (ky + ty), n, X, r, v);
                if (ty > 0 && ky - ty >= 0)
                    sym_row<Acc>(D, pl * z + (int64_t)n * (ky - ty), n, X, r, v);
            }
        }
    }
}

// inclusive prefix sums along every row of n entries, in place (a warp per row, 32-entry
// pages scanned with shuffles, the eight loads of a 256-entry stretch issued together)
template <typename Acc>
__global__ void __launch_bounds__(256) k_sym_rowscan(Acc *D, int n, int64_t rows)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row >= rows) return;
    Acc *r = D + row * n;
    Acc carry = 0;
    for (int p0 = 0; p0 < n; p0 += 256) {
        Acc v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int x = p0 + 32 * q + lane;
            v[q] = x < n ? r[x] : (Acc)0;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            Acc s = v[q];
            for (int o = 1; o < 32; o <<= 1) {
                const Acc t = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += t;
            }
            s += carry;
            const int x = p0 + 32 * q + lane;
            if (x < n) r[x] = s;
            carry = __shfl_sync(0xffffffffu, s, 31);
        }
    }
}

// L u = (half1 + half2) / 2, half1 already in Lu
__global__ void k_sym_finish_f32(SymArgs a, const float *__restrict__ u, float *__restrict__ Lu,
                                 const long long *__restrict__ S, const unsigned int *mx)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int sh = sym_shift_of(a.N, mx);
    const double s2 = __longlong_as_double((long long)(sh + 1023) << 52);     // 2^sh
    const double t = (double)u[i] * a.T[i] * s2;
    float h2;
    if (fabs(t) < 0x1p62) {
        const long long D2 = S[i] - __double2ll_rn(t);
        h2 = ldexpf(a.G32[i] * (float)D2, -sh);
    } else {
        h2 = (float)(a.G64[i] * (ldexp((double)S[i], -sh) - (double)u[i] * a.T[i]));
    }
    Lu[i] = 0.5f * (Lu[i] + h2);
}

__global__ void k_sym_finish_f64(SymArgs a, const double *__restrict__ u, double *__restrict__ Lu,
                                 const double *__restrict__ S)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    Lu[i] = 0.5 * (Lu[i] + a.G64[i] * (S[i] - u[i] * a.T[i]));
}

__global__ void k_sym_absmax_parts(int64_t N, const float *__restrict__ u,
                                   const float *__restrict__ c, float *__restrict__ part)
{
    __shared__ float s_w[8];
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(u[i] * c[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmaxf(m, s_w[w]);
        part[blockIdx.x] = m * (1.f + 0x1p-20f);
    }
}

__global__ void k_sym_copy_diag(int64_t N, const double *__restrict__ src, double *__restrict__ dst)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) dst[i] = src[i];
}

// ---------------------------------------------------------------------------
// K >= 1: the transpose half with the weights p(|o|^2 / R_k^2) of the source node k.  Along a
// leaf row of k's leaf set (node offsets o_y, o_z fixed, E = o_y^2 + o_z^2) the weight of the
// target column x is
//   sum_m f_m (E + (x - k_x)^2)^m,   f_m = c_k u_k p_m / R_k^{2m},
// a polynomial of degree 2K in x.  Each f_m, scaled by 2^S', is rounded once to an integer
// held in two limbs, H 2^B + Lo (0 <= Lo <= 2^B); the coefficients of the polynomial in x are
// then integer combinations of the limbs (binomials, powers of E and -k_x), exact modulo 2^64,
// and go into per-row difference arrays (+ at the run's first cell, - one past its last) of the
// 2K + 1 powers of x and the two limbs.  After the row prefix sums, the target i evaluates
// sum_e P_e(i) i_x^e per limb, again modulo 2^64: each limb's total is a sum of small
// weights times bounded integers and fits 63 bits, so both come out exact and
//   S_i = (H-total 2^B + Lo-total) 2^-S'.
// The order of the atomics cannot change a bit.  FP32 data keep the H limb alone (B = 0: one
// rounding of ~2^-28 of the largest term, far below FP32), FP64 data both.
// ---------------------------------------------------------------------------
struct SymKArgs {
    int n, K, limb, lgc, two;         // two: H and Lo limbs (FP64 data); else H alone, B = 0
    int64_t N;
    double p[8];
    const int *thr4;
    const double *c64, *ir2;
    long long *P;                     // plane (e, limb): P + (2 e + limb) N
    const unsigned int *mx;           // bound of max |c u| (FP32 bits)
};

// S' = S_H + B, S_H = 62 - lgc - e1 with max |c u| < 2^e1 and 2^lgc >= sources per target x
// the weight bound
__device__ __forceinline__ int symk_shift(const SymKArgs &a)
{
    const float m = __uint_as_float(*a.mx);
    int e1 = 0;
    if (m > 0.f) frexpf(m, &e1);
    return 62 - a.lgc - e1 + (a.two ? a.limb : 0);
}

__device__ __forceinline__ unsigned long long symk_binom(int m, int j)
{
    unsigned long long b = 1ull;
    for (int z = 0; z < j; ++z) b = b * (unsigned long long)(m - z) / (unsigned long long)(z + 1);
    return b;
}

template <int K, bool TWO>
__device__ __forceinline__ void symk_row(const SymKArgs &a, int64_t rowoff, int X, int r,
                                         int kx, int E, const unsigned long long (&FH)[K + 1],
                                         const unsigned long long (&FL)[K + 1])
{
    typedef unsigned long long u64;
    const int n = a.n;
    const int ka = max(0, -((r - X) >> 1) - 1);
    const int kb = min(n - 1, (X + r) >> 1);
    if (ka > kb) return;
    u64 nk[2 * K + 1], Ep[K + 1];
    nk[0] = 1ull;
    for (int q = 1; q <= 2 * K; ++q) nk[q] = nk[q - 1] * (u64)(-(long long)kx);
    Ep[0] = 1ull;
    for (int q = 1; q <= K; ++q) Ep[q] = Ep[q - 1] * (u64)E;
    u64 AH[2 * K + 1], AL[2 * K + 1];
#pragma unroll
    for (int e = 0; e <= 2 * K; ++e) { AH[e] = 0ull; AL[e] = 0ull; }
#pragma unroll
    for (int m = 0; m <= K; ++m)
#pragma unroll
        for (int j = 0; j <= m; ++j) {
            const u64 c1 = symk_binom(m, j) * Ep[m - j];
#pragma unroll
            for (int e = 0; e <= 2 * j; ++e) {
                const u64 c = c1 * symk_binom(2 * j, e) * nk[2 * j - e];
                AH[e] += FH[m] * c;
                if (TWO) AL[e] += FL[m] * c;
            }
        }
    const int64_t N = a.N;
    constexpr int LS = TWO ? 2 : 1;             // planes per power of x
    unsigned long long *P = reinterpret_cast<unsigned long long *>(a.P);
#pragma unroll
    for (int e = 0; e <= 2 * K; ++e) {
        atomicAdd(P + (LS * e) * N + rowoff + ka, AH[e]);
        if (TWO) atomicAdd(P + (2 * e + 1) * N + rowoff + ka, AL[e]);
        if (kb + 1 < n) {
            atomicAdd(P + (LS * e) * N + rowoff + kb + 1, 0ull - AH[e]);
            if (TWO) atomicAdd(P + (2 * e + 1) * N + rowoff + kb + 1, 0ull - AL[e]);
        }
    }
}

template <int DIM, int K, typename T, bool TWO>
__global__ void __launch_bounds__(256) k_symk_scatter(SymKArgs a, const T *__restrict__ u)
{
    typedef unsigned long long u64;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= a.N) return;
    const double v = a.c64[k] * (double)u[k];
    if (v == 0.0) return;
    const int sh = symk_shift(a);
    const double ir2 = a.ir2[k];
    u64 FH[K + 1], FL[K + 1];
    double pw = 1.0;
#pragma unroll
    for (int m = 0; m <= K; ++m) {
        const double y = ldexp(v * a.p[m] * pw, sh);
        if (TWO) {
            const double hi = floor(ldexp(y, -a.limb));
            FH[m] = (u64)(long long)hi;
            FL[m] = (u64)llrint(y - ldexp(hi, a.limb));
        } else {
            FH[m] = (u64)llrint(y);
            FL[m] = 0ull;
        }
        pw *= ir2;
    }
    const int n = a.n;
    const int kx = (int)(k % n);
    const int ky = DIM > 1 ? (int)((k / n) % n) : 0;
    const int kz = DIM > 2 ? (int)(k / ((int64_t)n * n)) : 0;
    const int X = 2 * kx + 1;
    const int T4 = a.thr4[k];
    if (DIM == 1) {
        symk_row<K, TWO>(a, 0, X, sym_isqrt(T4), kx, 0, FH, FL);
        return;
    }
    const int64_t pl = (int64_t)n * n;
    for (int tz = 0; tz <= (DIM > 2 ? n : 0); ++tz) {
        const int ez = tz == 0 ? 0 : sym_sq(2 * tz - 1);
        if (ez > T4) break;
        for (int sz = 0; sz < (DIM > 2 && tz > 0 ? 2 : 1); ++sz) {
            const int z = DIM > 2 ? (sz ? kz - tz : kz + tz) : 0;
            if (z < 0 || z >= (DIM > 2 ? n : 1)) continue;
            for (int ty = 0;; ++ty) {
                const int e = ez + (ty == 0 ? 0 : sym_sq(2 * ty - 1));
                if (e > T4) break;
                const int r = sym_isqrt(T4 - e);
                const int E = ty * ty + tz * tz;
                if (ky + ty < n) symk_row<K, TWO>(a, pl * z + (int64_t)n * (ky + ty), X, r, kx, E, FH, FL);
                if (ty > 0 && ky - ty >= 0)
                    symk_row<K, TWO>(a, pl * z + (int64_t)n * (ky - ty), X, r, kx, E, FH, FL);
            }
        }
    }
}

// per-block bounds of |c u| (FP64 products, rounded up to FP32) and their maximum
template <typename T>
__global__ void __launch_bounds__(256) k_symk_absmax(int64_t N, const T *__restrict__ u,
                                                     const double *__restrict__ c,
                                                     float *__restrict__ part)
{
    __shared__ double s_w[8];
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(c[i] * (double)u[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmax(m, s_w[w]);
        part[blockIdx.x] = (float)m * (1.f + 0x1p-20f);
    }
}

__global__ void k_symk_reduce(const float *__restrict__ part, int nparts, unsigned int *mx)
{
    float m = 0.f;
    for (int k = threadIdx.x; k < nparts; k += 32) m = fmaxf(m, part[k]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) *mx = __float_as_uint(m);
}

// S_i from the prefix sums, then L u = (half1 + half2) / 2 with half2 = G_i (S_i - u_i T_i)
template <typename T>
__global__ void k_symk_finish(SymKArgs a, const double *__restrict__ G,
                              const double *__restrict__ Tsum, const T *__restrict__ u,
                              T *__restrict__ Lu)
{
    typedef unsigned long long u64;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const u64 x = (u64)(i % a.n);
    const u64 *P = reinterpret_cast<const u64 *>(a.P);
    const int ls = a.two ? 2 : 1;
    u64 SH = 0ull, SL = 0ull, xp = 1ull;
    for (int e = 0; e <= 2 * a.K; ++e) {
        SH += P[(ls * e) * a.N + i] * xp;
        if (a.two) SL += P[(2 * e + 1) * a.N + i] * xp;
        xp *= x;
    }
    const int sh = symk_shift(a);
    const double S = a.two ? ldexp((double)(long long)SH, a.limb - sh) +
                                 ldexp((double)(long long)SL, -sh)
                           : ldexp((double)(long long)SH, -sh);
    const double h2 = G[i] * (S - (double)u[i] * Tsum[i]);
    Lu[i] = (T)(0.5 * ((double)Lu[i] + h2));
}

template <typename T>
static nl_status symk_launch(nl_plan *p, const T *u, T *Lu, int nrhs, cudaStream_t st);

SymArgs make_sym_args(nl_plan *p)
{
    SymArgs a;
    a.d = p->d; a.n = p->n; a.coef = p->coef; a.N = p->N;
    a.sigma = p->sigma;
    a.hd = std::pow(p->h, (double)p->d);
    a.thr4 = p->thr4;
    a.delta = nullptr; a.acoef = nullptr;
    a.c64 = p->sym_c64; a.c32 = p->sym_c32; a.T = p->sym_T;
    a.G64 = p->sym_G64; a.G32 = p->sym_G32; a.diag = p->sym_diag;
    a.fastF = p->fastF; a.selfS = p->selfS;
    a.K = p->K;
    for (int m = 0; m < 8; ++m) a.p[m] = p->poly[m];
    a.ir2 = p->sym_ir2;
    return a;
}

SymKArgs make_symk_args(nl_plan *p)
{
    SymKArgs a;
    a.n = p->n; a.K = p->K; a.limb = p->sym_limb; a.lgc = p->sym_lgc; a.N = p->N; a.two = 1;
    for (int m = 0; m < 8; ++m) a.p[m] = p->poly[m];
    a.thr4 = p->thr4; a.c64 = p->sym_c64; a.ir2 = p->sym_ir2; a.P = p->sym_P;
    a.mx = (const unsigned int *)p->sym_aux;
    return a;
}

template <typename T>
static nl_status symk_launch(nl_plan *p, const T *u, T *Lu, int nrhs, cudaStream_t st)
{
    const int64_t N = p->N;
    const int d = p->d, n = p->n, K = p->K;
    SymKArgs a = make_symk_args(p);
    // FP32 data: one limb (its rounding, ~2^-28 of the largest term, is far below FP32);
    // FP64 data: two
    constexpr bool TWO = sizeof(T) == 8;
    a.two = TWO ? 1 : 0;
    const unsigned gb = (unsigned)((N + 255) / 256);
    const int64_t rows = N / n;
    const unsigned gr = (unsigned)((rows * 32 + 255) / 256);
    unsigned int *mx = (unsigned int *)p->sym_aux;
    float *part = (float *)(p->sym_aux + 16);
    int64_t per = (N + NL_FAST_PARTS - 1) / NL_FAST_PARTS;
    if (per < 2048) per = 2048;
    const int nparts = (int)((N + per - 1) / per);
    const int planes = (TWO ? 2 : 1) * (2 * K + 1);
    for (int r = 0; r < nrhs; ++r) {
        const T *ur = u + r * N;
        T *lr = Lu + r * N;
        NL_CUDA_TRY(cudaMemsetAsync(p->sym_P, 0, (size_t)planes * N * sizeof(long long), st));
        k_symk_absmax<T><<<nparts, 256, 0, st>>>(N, ur, p->sym_c64, part);
        k_symk_reduce<<<1, 32, 0, st>>>(part, nparts, mx);
#define NL_SYMK(DD, KK) k_symk_scatter<DD, KK, T, TWO><<<gb, 256, 0, st>>>(a, ur)
        if (d == 1) {
            if (K == 1) NL_SYMK(1, 1); else if (K == 2) NL_SYMK(1, 2); else NL_SYMK(1, 3);
        } else if (d == 2) {
            if (K == 1) NL_SYMK(2, 1); else if (K == 2) NL_SYMK(2, 2); else NL_SYMK(2, 3);
        } else {
            if (K == 1) NL_SYMK(3, 1); else if (K == 2) NL_SYMK(3, 2); else NL_SYMK(3, 3);
        }
#undef NL_SYMK
        for (int q = 0; q < planes; ++q)
            k_sym_rowscan<long long><<<gr, 256, 0, st>>>(p->sym_P + (int64_t)q * N, n, rows);
        k_symk_finish<T><<<gb, 256, 0, st>>>(a, p->sym_G64, p->sym_T, ur, lr);
        NL_CUDA_TRY(cudaGetLastError());
    }
    return NL_OK;
}

}  // namespace

nl_status nl_fast_sym_plan_init(nl_plan *p, const double *delta_dev, const double *a_dev,
                                cudaStream_t st)
{
    const int64_t N = p->N;
    auto alloc = [&](void **ptr, size_t bytes) -> nl_status {
        if (cudaMalloc(ptr, bytes ? bytes : 1) != cudaSuccess) {
            nl_set_error("cudaMalloc(%zu) for the symmetrised fast path failed", bytes);
            return NL_ENOMEM;
        }
        p->device_bytes += bytes;
        return NL_OK;
    };
    nl_status s;
    if ((s = alloc((void **)&p->sym_c64, N * sizeof(double))) != NL_OK) return s;
    if ((s = alloc((void **)&p->sym_c32, N * sizeof(float))) != NL_OK) return s;
    if ((s = alloc((void **)&p->sym_T, N * sizeof(double))) != NL_OK) return s;
    if ((s = alloc((void **)&p->sym_G64, N * sizeof(double))) != NL_OK) return s;
    if ((s = alloc((void **)&p->sym_G32, N * sizeof(float))) != NL_OK) return s;
    if ((s = alloc((void **)&p->sym_diag, N * sizeof(double))) != NL_OK) return s;
    if ((s = alloc((void **)&p->sym_D, N * sizeof(double))) != NL_OK) return s;
    if ((s = alloc((void **)&p->sym_aux, 16 + NL_FAST_PARTS * sizeof(float))) != NL_OK) return s;
    if (p->K >= 1) {
        // sources reaching a target: at most (2 Rmax + 3)^d; |o|^2 / R_k^2 < (1 + sqrt(d) /
        // (2 R_min))^2 on a leaf set, so |p| <= sum_m |p_m| rho^m; |o|^2 <= d (Rmax + 1)^2
        const int d = p->d;
        const double count = std::pow(2.0 * p->Rmax + 3.0, (double)d);
        const double rr = 1.0 + std::sqrt((double)d) / (2.0 * std::max(p->rho_min, 1e-3));
        double pb = 0.0, rp = 1.0;
        for (int m = 0; m <= p->K; ++m) { pb += std::fabs(p->poly[m]) * rp; rp *= rr * rr; }
        const double omax2 = d * (p->Rmax + 1.0) * (p->Rmax + 1.0);
        const double lbound = count * (p->K + 1) * std::pow(omax2, (double)p->K);
        p->sym_lgc = (int)std::ceil(std::log2(count * pb));
        p->sym_limb = 62 - (int)std::ceil(std::log2(lbound));
        if (p->sym_limb < 8 || p->sym_lgc > 40) {
            nl_set_error("nl_plan_create: the symmetric NL_POLY variant with K >= 1 needs a "
                         "smaller horizon (integer sums beyond 64 bits)");
            return NL_EUNSUPPORTED;
        }
        if ((s = alloc((void **)&p->sym_ir2, N * sizeof(double))) != NL_OK) return s;
        if ((s = alloc((void **)&p->sym_P, (size_t)2 * (2 * p->K + 1) * N * sizeof(long long))) != NL_OK)
            return s;
    }
    SymArgs a = make_sym_args(p);
    a.delta = delta_dev;
    a.acoef = a_dev;
    const unsigned gb = (unsigned)((N + 255) / 256);
    k_sym_coef<<<gb, 256, 0, st>>>(a);
    k_sym_node<<<gb, 256, 0, st>>>(a, p->Rmax + 1);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

nl_status nl_fast_sym_diag(nl_plan *p, double *diag, cudaStream_t st)
{
    k_sym_copy_diag<<<(unsigned)((p->N + 255) / 256), 256, 0, st>>>(p->N, p->sym_diag, diag);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

// half1 by the one-sided fast apply (any route), then per right-hand side the scatter, the row
// prefix sums and the combination
nl_status nl_fast_sym_launch(nl_plan *p, const void *u, void *Lu, int nrhs, int dtype,
                             cudaStream_t st)
{
    nl_status s = nl_fast_launch(p, u, Lu, nrhs, dtype, st);
    if (s != NL_OK) return s;
    if (p->K >= 1) {
        if (dtype == NL_F32) return symk_launch<float>(p, (const float *)u, (float *)Lu, nrhs, st);
        return symk_launch<double>(p, (const double *)u, (double *)Lu, nrhs, st);
    }
    const int64_t N = p->N;
    const int d = p->d, n = p->n;
    SymArgs a = make_sym_args(p);
    const unsigned gb = (unsigned)((N + 255) / 256);
    const int64_t rows = N / n;
    const unsigned gr = (unsigned)((rows * 32 + 255) / 256);
    unsigned int *mx = (unsigned int *)p->sym_aux;
    float *part = (float *)(p->sym_aux + 16);
    int64_t per = (N + NL_FAST_PARTS - 1) / NL_FAST_PARTS;
    if (per < 2048) per = 2048;
    const int nparts = (int)((N + per - 1) / per);
    for (int r = 0; r < nrhs; ++r) {
        NL_CUDA_TRY(cudaMemsetAsync(p->sym_D, 0, N * sizeof(double), st));
        if (dtype == NL_F32) {
            const float *ur = (const float *)u + r * N;
            float *lr = (float *)Lu + r * N;
            long long *D = (long long *)p->sym_D;
            k_sym_absmax_parts<<<nparts, 256, 0, st>>>(N, ur, p->sym_c32, part);
            if (d == 1) k_sym_scatter<1, float, long long><<<gb, 256, 0, st>>>(a, ur, D, part, nparts, mx);
            else if (d == 2) k_sym_scatter<2, float, long long><<<gb, 256, 0, st>>>(a, ur, D, part, nparts, mx);
            else k_sym_scatter<3, float, long long><<<gb, 256, 0, st>>>(a, ur, D, part, nparts, mx);
            k_sym_rowscan<long long><<<gr, 256, 0, st>>>(D, n, rows);
            k_sym_finish_f32<<<gb, 256, 0, st>>>(a, ur, lr, D, mx);
        } else {
            const double *ur = (const double *)u + r * N;
            double *lr = (double *)Lu + r * N;
            double *D = p->sym_D;
            if (d == 1) k_sym_scatter<1, double, double><<<gb, 256, 0, st>>>(a, ur, D, nullptr, 0, nullptr);
            else if (d == 2) k_sym_scatter<2, double, double><<<gb, 256, 0, st>>>(a, ur, D, nullptr, 0, nullptr);
            else k_sym_scatter<3, double, double><<<gb, 256, 0, st>>>(a, ur, D, nullptr, 0, nullptr);
            k_sym_rowscan<double><<<gr, 256, 0, st>>>(D, n, rows);
            k_sym_finish_f64<<<gb, 256, 0, st>>>(a, ur, lr, D);
        }
        NL_CUDA_TRY(cudaGetLastError());
    }
    return NL_OK;
}
