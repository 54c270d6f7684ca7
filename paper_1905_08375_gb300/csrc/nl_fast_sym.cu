// nl_fast_sym.cu -- the fast path for the symmetrised (divergence-type) polynomial operator,
// K = 0 (a project extension of Sec. 3, which treats the one-sided C(x) delta(x) form only;
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
    int d, n, coef;
    int64_t N;
    double sigma, hd;
    const int *thr4;
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
}

// Plan time, per node i: T_i by the definition -- every cell k of the box of radius B around i
// whose own leaf set reaches i (the half-unit gap from node k to cell i, per axis 2|o| - 1, 0
// for o = 0, squared and summed, at most thr4_k; cells outside Omega take the node's own
// horizon and coefficient, so there the test is the node's own) -- and the Jacobi diagonal
//   -L_ii = [fastF_i (selfS_i - h^d b_i) + G_i (T_i - c_i)] / 2.
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
            for (int ox = -B; ox <= B; ++ox) {
                const int gx = ox ? 2 * abs(ox) - 1 : 0;
                const int e = gx * gx + eyz;
                const int kx = ix + ox;
                if (iny && kx >= 0 && kx < n) {
                    const int64_t k = kx + (int64_t)n * (ky + (int64_t)n * kz);
                    if (e <= a.thr4[k]) T += a.c64[k];
                } else if (e <= T4i) {
                    T += ci;
                }
            }
        }
    }
    const double ai = a.coef == NL_COEF_XY ? a.acoef[i] : 1.0;
    a.T[i] = T;
    a.diag[i] = 0.5 * (a.fastF[i] * (a.selfS[i] - a.hd * ai) + a.G64[i] * (T - ci));
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
    return a;
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
