// nl_direct.cu -- the direct variable-stencil apply ("Original" product of
// Sec. 2 and Sec. 4): Eq. (2.1)-(2.2) for scalar diffusion and Eq. (1.2) for
// linear bond-based peridynamics.
//
// Layout: one thread per output node, x fastest.  Each block stages the halo
// tile (block extent + 2 Rmax per dimension) of (u, b) -- or (u, b, W/2, thr)
// for the symmetric variant, (ux, uy, c, inside) for peridynamics -- in shared
// memory, then walks the offset table of the ball, sorted by |o|^2, so that a
// node with threshold thr_i reads exactly the prefix of cnt_i entries: the
// ragged per-node horizon costs nothing beyond its own ball.  Table entries
// are warp-uniform (broadcast loads); tile reads are consecutive in x across a
// warp (conflict-free).
#include <mutex>

#include "nl_internal.cuh"

template <typename T> struct V2 { T u, b; };
template <typename T> struct V4 { T u, b, wh; int thr; };
template <typename T> struct PdV { T ux, uy, c, in; };

template <typename T> struct Tab;
template <> struct Tab<float> { using type = OffEntry32; using pd = PdEntry32; };
template <> struct Tab<double> { using type = OffEntry64; using pd = PdEntry64; };

struct DirectArgs {
    int n, R, sx, sy, sz, K;
    int64_t N;
    const int *cnt, *thr;
    const void *b, *fin, *ext, *wh, *ir;
    const void *tab;
    const int4 *off;
    double poly[8];
    double pd_scale;
    const double *pdext;
};

enum { MODE_POWER = 0, MODE_POLY = 1, MODE_SYM = 2 };

template <int D>
__device__ __forceinline__ void block_origin(int n, int &x0, int &y0, int &z0)
{
    constexpr int BX = DirectBlock<D>::X, BY = DirectBlock<D>::Y, BZ = DirectBlock<D>::Z;
    x0 = blockIdx.x * BX;
    y0 = 0; z0 = 0;
    if (D > 1) {
        const int tiles_y = (n + BY - 1) / BY;
        y0 = (blockIdx.y % tiles_y) * BY;
        if (D > 2) z0 = (blockIdx.y / tiles_y) * BZ;
    }
}

template <int D>
__device__ __forceinline__ bool in_grid(int n, int x, int y, int z)
{
    bool ok = (unsigned)x < (unsigned)n;
    if (D > 1) ok = ok && (unsigned)y < (unsigned)n;
    if (D > 2) ok = ok && (unsigned)z < (unsigned)n;
    return ok;
}

template <typename T>
__device__ __forceinline__ T poly_weight(const double *pc, int K, T t)
{
    T r = (T)pc[K];
    for (int m = K - 1; m >= 0; --m) r = r * t + (T)pc[m];
    return r;
}

// ---------------------------------------------------------------------------
// scalar kernel
// ---------------------------------------------------------------------------
// DIAG = true writes the diagonal of -L instead: fin_i (sum_o wgt(o) + ext_i).
template <int D, typename T, int MODE, bool STAGE, bool DIAG = false>
__global__ void __launch_bounds__(DirectBlock<D>::X * DirectBlock<D>::Y * DirectBlock<D>::Z)
k_direct_scalar(DirectArgs a, const T *__restrict__ u, T *__restrict__ Lu)
{
    constexpr int BX = DirectBlock<D>::X, BY = DirectBlock<D>::Y, BZ = DirectBlock<D>::Z;
    using Elem = typename std::conditional<MODE == MODE_SYM, V4<T>, V2<T>>::type;
    using Entry = typename Tab<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Elem *tile = reinterpret_cast<Elem *>(smem_raw);

    const int n = a.n, R = a.R;
    const int64_t N = a.N;
    const T *__restrict__ ur = u + (int64_t)blockIdx.z * N;
    const T *__restrict__ bb = (const T *)a.b;
    const T *__restrict__ whv = (const T *)a.wh;
    int x0, y0, z0;
    block_origin<D>(n, x0, y0, z0);

    if (STAGE) {
        const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
        const int elems = a.sx * a.sy * a.sz;
        for (int e = tid; e < elems; e += BX * BY * BZ) {
            const int ex = e % a.sx;
            const int ey = (e / a.sx) % a.sy;
            const int ez = e / (a.sx * a.sy);
            const int gx = x0 - R + ex;
            const int gy = D > 1 ? y0 - R + ey : 0;
            const int gz = D > 2 ? z0 - R + ez : 0;
            Elem v;
            if (in_grid<D>(n, gx, gy, gz)) {
                const int64_t j = gx + (int64_t)n * (gy + (int64_t)n * gz);
                v.u = ur[j];
                v.b = bb[j];
                if constexpr (MODE == MODE_SYM) { v.wh = whv[j]; v.thr = a.thr[j]; }
            } else {
                v.u = T(0);
                v.b = T(0);
                if constexpr (MODE == MODE_SYM) { v.wh = T(0); v.thr = -1; }
            }
            tile[e] = v;
        }
        __syncthreads();
    }

    const int x = x0 + threadIdx.x;
    const int y = D > 1 ? y0 + threadIdx.y : 0;
    const int z = D > 2 ? z0 + threadIdx.z : 0;
    if (!in_grid<D>(n, x, y, z)) return;
    const int64_t i = x + (int64_t)n * (y + (int64_t)n * z);
    const T ui = ur[i];
    const int cnt = a.cnt[i];
    const Entry *__restrict__ tab = (const Entry *)a.tab;

    int centre = 0;
    if (STAGE) {
        centre = (threadIdx.x + R);
        if (D > 1) centre += a.sx * (threadIdx.y + R);
        if (D > 2) centre += a.sx * a.sy * (threadIdx.z + R);
    }
    T ir = T(0), whi = T(0);
    int thri = 0;
    if constexpr (MODE == MODE_POLY) ir = ((const T *)a.ir)[i];
    if constexpr (MODE == MODE_SYM) { whi = whv[i]; thri = a.thr[i]; }

    T acc0 = T(0), acc1 = T(0);
#pragma unroll 2
    for (int t = 0; t < cnt; ++t) {
        const Entry en = tab[t];
        T uj, bj, whj = T(0);
        int thrj = -1;
        if (STAGE) {
            const Elem v = tile[centre + en.soff];
            uj = v.u; bj = v.b;
            if constexpr (MODE == MODE_SYM) { whj = v.wh; thrj = v.thr; }
        } else {
            const int4 o = a.off[t];
            const int gx = x + o.x, gy = y + o.y, gz = z + o.z;
            if (in_grid<D>(n, gx, gy, gz)) {
                const int64_t j = gx + (int64_t)n * (gy + (int64_t)n * gz);
                uj = ur[j]; bj = bb[j];
                if constexpr (MODE == MODE_SYM) { whj = whv[j]; thrj = a.thr[j]; }
            } else {
                uj = T(0); bj = T(0);
            }
        }
        T w;
        if constexpr (MODE == MODE_POWER) {
            w = (T)en.g * bj;
        } else if constexpr (MODE == MODE_POLY) {
            w = poly_weight<T>(a.poly, a.K, (T)en.o2 * ir) * bj;
        } else {
            const T wi = (en.o2 <= thri) ? whi : T(0);
            const T wj = (en.o2 <= thrj) ? whj : T(0);
            w = (T)en.g * bj * (wi + wj);
        }
        const T term = DIAG ? w : w * (uj - ui);
        if (t & 1) acc1 += term; else acc0 += term;
    }
    const T fin = ((const T *)a.fin)[i];
    const T ext = ((const T *)a.ext)[i];
    if (DIAG)
        Lu[(int64_t)blockIdx.z * N + i] = fin * ((acc0 + acc1) + ext);
    else
        Lu[(int64_t)blockIdx.z * N + i] = fin * ((acc0 + acc1) - ui * ext);
}

// ---------------------------------------------------------------------------
// peridynamic kernel (d = 2): acc = sum (c_i in_j + c_j) G(o) (u_j - u_i);
// Lu = sigma h^{d-1} (acc/2 - E_i u_i), E_i = c_i sum_{exterior o} G(o).
// FP32: FP32 products, FP32 partial sums over 32 bonds, FP64 running sum.
// ---------------------------------------------------------------------------
// DIAG = true writes the per-component diagonal of -L_PD instead.
template <typename T, bool STAGE, bool DIAG = false>
__global__ void __launch_bounds__(256)
k_direct_pd(DirectArgs a, const T *__restrict__ u, T *__restrict__ Lu)
{
    constexpr int BX = DirectBlock<2>::X, BY = DirectBlock<2>::Y;
    using Entry = typename Tab<T>::pd;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PdV<T> *tile = reinterpret_cast<PdV<T> *>(smem_raw);
    const int n = a.n, R = a.R;
    const int64_t N = a.N;
    const T *__restrict__ ux = u + (int64_t)blockIdx.z * 2 * N;
    const T *__restrict__ uy = ux + N;
    const T *__restrict__ cc = (const T *)a.b;
    int x0, y0, z0;
    block_origin<2>(n, x0, y0, z0);
    if (STAGE) {
        const int tid = threadIdx.x + BX * threadIdx.y;
        const int elems = a.sx * a.sy;
        for (int e = tid; e < elems; e += BX * BY) {
            const int gx = x0 - R + e % a.sx;
            const int gy = y0 - R + e / a.sx;
            PdV<T> v;
            if (in_grid<2>(n, gx, gy, 0)) {
                const int64_t j = gx + (int64_t)n * gy;
                v.ux = ux[j]; v.uy = uy[j]; v.c = cc[j]; v.in = T(1);
            } else {
                v.ux = T(0); v.uy = T(0); v.c = T(0); v.in = T(0);
            }
            tile[e] = v;
        }
        __syncthreads();
    }
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (!in_grid<2>(n, x, y, 0)) return;
    const int64_t i = x + (int64_t)n * y;
    const T uxi = ux[i], uyi = uy[i], ci = cc[i];
    const int cnt = a.cnt[i];
    const Entry *__restrict__ tab = (const Entry *)a.tab;
    const int centre = (threadIdx.x + R) + a.sx * (threadIdx.y + R);
    double sx = 0.0, sy = 0.0;
    T px = T(0), py = T(0);
    for (int t = 0; t < cnt; ++t) {
        const Entry en = tab[t];
        T uxj, uyj, cj, inj;
        if (STAGE) {
            const PdV<T> v = tile[centre + en.soff];
            uxj = v.ux; uyj = v.uy; cj = v.c; inj = v.in;
        } else {
            const int4 o = a.off[t];
            const int gx = x + o.x, gy = y + o.y;
            if (in_grid<2>(n, gx, gy, 0)) {
                const int64_t j = gx + (int64_t)n * gy;
                uxj = ux[j]; uyj = uy[j]; cj = cc[j]; inj = T(1);
            } else {
                uxj = T(0); uyj = T(0); cj = T(0); inj = T(0);
            }
        }
        const T w = ci * inj + cj;
        if (DIAG) {
            px += w * (T)en.gxx;
            py += w * (T)en.gyy;
        } else {
            const T dx = uxj - uxi, dy = uyj - uyi;
            px += w * ((T)en.gxx * dx + (T)en.gxy * dy);
            py += w * ((T)en.gxy * dx + (T)en.gyy * dy);
        }
        if ((t & 31) == 31) { sx += (double)px; sy += (double)py; px = T(0); py = T(0); }
    }
    sx += (double)px;
    sy += (double)py;
    const double *E = a.pdext + 3 * i;
    double ox, oy;
    if (DIAG) {
        ox = a.pd_scale * (0.5 * sx + E[0]);
        oy = a.pd_scale * (0.5 * sy + E[2]);
    } else {
        ox = a.pd_scale * (0.5 * sx - (E[0] * (double)uxi + E[1] * (double)uyi));
        oy = a.pd_scale * (0.5 * sy - (E[1] * (double)uxi + E[2] * (double)uyi));
    }
    T *out = Lu + (int64_t)blockIdx.z * 2 * N;
    out[i] = (T)ox;
    out[N + i] = (T)oy;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// Raise a kernel's dynamic shared-memory limit once per (kernel, size): repeated calls
// (and calls while a stream is being captured) then issue no runtime call at all.
static std::mutex g_smem_mu;
static const void *g_smem_fn[256];
static size_t g_smem_bytes[256];
static int g_smem_count = 0;

template <typename K>
static cudaError_t prep_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    const void *key = (const void *)kernel;
    std::lock_guard<std::mutex> lock(g_smem_mu);
    int slot = -1;
    for (int k = 0; k < g_smem_count; ++k)
        if (g_smem_fn[k] == key) { slot = k; break; }
    if (slot >= 0 && g_smem_bytes[slot] >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    if (slot < 0 && g_smem_count < 256) { slot = g_smem_count++; g_smem_fn[slot] = key; }
    if (slot >= 0) g_smem_bytes[slot] = bytes;
    return e;
}

template <int D>
static dim3 direct_grid(int n, int nrhs)
{
    constexpr int BX = DirectBlock<D>::X, BY = DirectBlock<D>::Y, BZ = DirectBlock<D>::Z;
    unsigned gx = (n + BX - 1) / BX;
    unsigned gy = 1;
    if (D > 1) gy = (n + BY - 1) / BY;
    if (D > 2) gy *= (n + BZ - 1) / BZ;
    return dim3(gx, gy, nrhs);
}

template <int D, typename T, int MODE>
static nl_status launch_scalar_t(nl_plan *p, const DirectArgs &a, const T *u, T *Lu, int nrhs,
                                 cudaStream_t st, size_t smem)
{
    const dim3 blk(DirectBlock<D>::X, DirectBlock<D>::Y, DirectBlock<D>::Z);
    const dim3 grd = direct_grid<D>(p->n, nrhs);
    if (p->stage) {
        auto kern = k_direct_scalar<D, T, MODE, true>;
        NL_CUDA_TRY(prep_smem(kern, smem));
        kern<<<grd, blk, smem, st>>>(a, u, Lu);
    } else {
        auto kern = k_direct_scalar<D, T, MODE, false>;
        kern<<<grd, blk, 0, st>>>(a, u, Lu);
    }
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

template <typename T>
static nl_status launch_scalar(nl_plan *p, const DirectArgs &a, const T *u, T *Lu, int nrhs,
                               cudaStream_t st, size_t smem)
{
    const int mode = p->symmetric ? MODE_SYM : (p->family == NL_POLY ? MODE_POLY : MODE_POWER);
#define NL_DISPATCH_MODE(D)                                                                  \
    do {                                                                                     \
        if (mode == MODE_POWER) return launch_scalar_t<D, T, MODE_POWER>(p, a, u, Lu, nrhs, st, smem); \
        if (mode == MODE_POLY) return launch_scalar_t<D, T, MODE_POLY>(p, a, u, Lu, nrhs, st, smem);   \
        return launch_scalar_t<D, T, MODE_SYM>(p, a, u, Lu, nrhs, st, smem);                 \
    } while (0)
    if (p->d == 1) NL_DISPATCH_MODE(1);
    if (p->d == 2) NL_DISPATCH_MODE(2);
    NL_DISPATCH_MODE(3);
#undef NL_DISPATCH_MODE
}

template <typename T>
static nl_status launch_pd(nl_plan *p, const DirectArgs &a, const T *u, T *Lu, int nrhs,
                           cudaStream_t st, size_t smem)
{
    const dim3 blk(DirectBlock<2>::X, DirectBlock<2>::Y, 1);
    const dim3 grd = direct_grid<2>(p->n, nrhs);
    if (p->stage) {
        auto kern = k_direct_pd<T, true>;
        NL_CUDA_TRY(prep_smem(kern, smem));
        kern<<<grd, blk, smem, st>>>(a, u, Lu);
    } else {
        k_direct_pd<T, false><<<grd, blk, 0, st>>>(a, u, Lu);
    }
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

static DirectArgs make_args(const nl_plan *p, int dtype)
{
    DirectArgs a;
    a.n = p->n; a.R = p->Rmax; a.sx = p->tile_sx; a.sy = p->tile_sy; a.sz = p->tile_sz;
    a.K = p->K; a.N = p->N;
    a.cnt = p->cnt; a.thr = p->thr;
    const bool f32 = dtype == NL_F32;
    a.b = f32 ? (const void *)p->b32 : (const void *)p->b64;
    a.fin = f32 ? (const void *)p->fin32 : (const void *)p->fin64;
    a.ext = f32 ? (const void *)p->ext32 : (const void *)p->ext64;
    a.wh = f32 ? (const void *)p->wh32 : (const void *)p->wh64;
    a.ir = f32 ? (const void *)p->ir32 : (const void *)p->ir64;
    if (p->family == NL_PD_BOND)
        a.tab = f32 ? (const void *)p->pd32 : (const void *)p->pd64;
    else
        a.tab = f32 ? (const void *)p->tab32 : (const void *)p->tab64;
    a.off = p->off;
    for (int m = 0; m < 8; ++m) a.poly[m] = p->poly[m];
    a.pd_scale = p->sigma * pow(p->h, p->d - 1.0);
    a.pdext = p->pdext;
    return a;
}

nl_status nl_direct_launch(nl_plan *p, const void *u, void *Lu, int nrhs, int dtype,
                           cudaStream_t st)
{
    const DirectArgs a = make_args(p, dtype);
    if (p->family == NL_PD_BOND) {
        if (dtype == NL_F32)
            return launch_pd<float>(p, a, (const float *)u, (float *)Lu, nrhs, st, p->smem_bytes32);
        return launch_pd<double>(p, a, (const double *)u, (double *)Lu, nrhs, st, p->smem_bytes64);
    }
    if (dtype == NL_F32)
        return launch_scalar<float>(p, a, (const float *)u, (float *)Lu, nrhs, st, p->smem_bytes32);
    return launch_scalar<double>(p, a, (const double *)u, (double *)Lu, nrhs, st, p->smem_bytes64);
}

template <int D>
static nl_status diag_scalar(nl_plan *p, const DirectArgs &a, const double *zin, double *diag,
                             cudaStream_t st)
{
    const dim3 blk(DirectBlock<D>::X, DirectBlock<D>::Y, DirectBlock<D>::Z);
    const dim3 grd = direct_grid<D>(p->n, 1);
    if (p->stage) {
        auto kern = k_direct_scalar<D, double, MODE_SYM, true, true>;
        NL_CUDA_TRY(prep_smem(kern, p->smem_bytes64));
        kern<<<grd, blk, p->smem_bytes64, st>>>(a, zin, diag);
    } else {
        k_direct_scalar<D, double, MODE_SYM, false, true><<<grd, blk, 0, st>>>(a, zin, diag);
    }
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

// Diagonal of -L (FP64), for the Jacobi preconditioner: [N] scalar, [2][N] peridynamic.
// `zin` is any readable input of the operator's length (its values are not used).
nl_status nl_diag_launch(nl_plan *p, const double *zin, double *diag, cudaStream_t st)
{
    const DirectArgs a = make_args(p, NL_F64);
    if (p->family == NL_PD_BOND) {
        const dim3 blk(DirectBlock<2>::X, DirectBlock<2>::Y, 1);
        const dim3 grd = direct_grid<2>(p->n, 1);
        if (p->stage) {
            auto kern = k_direct_pd<double, true, true>;
            NL_CUDA_TRY(prep_smem(kern, p->smem_bytes64));
            kern<<<grd, blk, p->smem_bytes64, st>>>(a, zin, diag);
        } else {
            k_direct_pd<double, false, true><<<grd, blk, 0, st>>>(a, zin, diag);
        }
        NL_CUDA_TRY(cudaGetLastError());
        return NL_OK;
    }
    if (!p->symmetric) {
        nl_set_error("diagonal: built for the symmetric scalar operator and peridynamics");
        return NL_EUNSUPPORTED;
    }
    if (p->d == 1) return diag_scalar<1>(p, a, zin, diag, st);
    if (p->d == 2) return diag_scalar<2>(p, a, zin, diag, st);
    return diag_scalar<3>(p, a, zin, diag, st);
}

extern "C" nl_status nl_apply(nl_plan *p, const void *u, void *Lu, int nrhs, int dtype,
                              void *stream)
{
    if (!nl_plan_ok(p)) {
        nl_set_error("nl_apply: invalid plan");
        return NL_EINVAL;
    }
    if (!u || !Lu || nrhs < 1 || nrhs > 65535 || (dtype != NL_F32 && dtype != NL_F64)) {
        nl_set_error("nl_apply: need non-null u/Lu, 1 <= nrhs <= 65535, dtype F32/F64");
        return NL_EINVAL;
    }
    return nl_direct_launch(p, u, Lu, nrhs, dtype, nl_stream(stream));
}
