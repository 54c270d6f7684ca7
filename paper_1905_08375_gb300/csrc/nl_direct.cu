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
#include <algorithm>
#include <mutex>
#include <vector>
#include <type_traits>

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
    const int *cnt_thr;       // symmetric variant: largest |o|^2 a node's loop must reach
    const void *b, *fin, *ext, *wh, *ir;
    const void *tab;
    const int4 *off;
    double poly[8];
    double pd_scale;
    const double *pdext;
    const float *pdg;         // PD, constant horizon: dense [2R+1][2R+1][3] bond tensors
    const double *skip;       // symmetric paired-column kernels inside CG: right-hand side z
    int skip_stride;          // needs no result when skip[z * skip_stride] != 0 (else null)
};

// MODE_KAPPA: the kappa part of the splitting of Sec. 3, weight ra_i |o|^{-alpha} - p(|o|^2/R2_i)
enum { MODE_POWER = 0, MODE_POLY = 1, MODE_SYM = 2, MODE_KAPPA = 3 };

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
    if constexpr (MODE == MODE_POLY || MODE == MODE_KAPPA) ir = ((const T *)a.ir)[i];
    if constexpr (MODE == MODE_SYM) { whi = whv[i]; thri = a.thr[i]; }
    if constexpr (MODE == MODE_KAPPA) whi = whv[i];           // ra_i = (delta_i / h)^alpha

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
        } else if constexpr (MODE == MODE_KAPPA) {
            w = ((T)en.g * whi - poly_weight<T>(a.poly, a.K, (T)en.o2 * ir)) * bj;
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
// 2-D register-blocked scalar kernel.  A block of 32 x RB_TY threads covers 32 columns and
// RB_TY * RB_P rows; each thread owns RB_P consecutive rows of one column.  The block stages
// its halo tile in shared memory (plus RB_P spare rows), then for every stencil column ox
// slides a register window down the tile: one shared load and one weight per row offset oy
// serve all RB_P outputs, each with its own exact horizon mask ox^2 + oy^2 <= thr_p.  The sum
// is accumulated column by column in the difference form g b_j (u_j - u_i).
// ---------------------------------------------------------------------------
constexpr int RB_TY = 4, RB_P = 8;

template <typename T, int MODE, int RP>
__global__ void __launch_bounds__(32 * RB_TY)
k_direct2d_rb(DirectArgs a, const T *__restrict__ gtab, const T *__restrict__ u, T *__restrict__ Lu)
{
    using Elem = typename std::conditional<MODE == MODE_SYM, V4<T>, V2<T>>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n, R = a.R;
    const int SX = 32 + 2 * R;                       // tile width
    const int SY = RB_TY * RP + 2 * R + RP;      // tile height (RP spare rows)
    const int GW = 2 * R + 1;
    Elem *tile = reinterpret_cast<Elem *>(smem_raw);
    T *s_g = reinterpret_cast<T *>(smem_raw + sizeof(Elem) * SX * SY);
    const int64_t N = a.N;
    const T *__restrict__ ur = u + (int64_t)blockIdx.z * N;
    const T *__restrict__ bb = (const T *)a.b;
    const T *__restrict__ whv = (const T *)a.wh;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * (RB_TY * RP);
    const int tid = threadIdx.x + 32 * threadIdx.y;
    for (int e = tid; e < SX * SY; e += 32 * RB_TY) {
        const int gx = x0 - R + e % SX, gy = y0 - R + e / SX;
        Elem v;
        if (gx >= 0 && gx < n && gy >= 0 && gy < n) {
            const int64_t j = gx + (int64_t)n * gy;
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
    if (MODE != MODE_POLY)
        for (int e = tid; e < GW * GW; e += 32 * RB_TY) s_g[e] = gtab[e];
    __syncthreads();

    const int x = x0 + threadIdx.x;
    const int ybase = y0 + threadIdx.y * RP;
    T ui[RP], acc[RP], irp[RP], whp[RP];
    int thr[RP];
    int tmax = -1;
#pragma unroll
    for (int p = 0; p < RP; ++p) {
        const int y = ybase + p;
        const bool own = x < n && y < n;
        const int64_t i = own ? x + (int64_t)n * y : 0;
        ui[p] = tile[(threadIdx.y * RP + p + R) * SX + threadIdx.x + R].u;
        thr[p] = own ? a.thr[i] : -1;
        irp[p] = (MODE == MODE_POLY && own) ? ((const T *)a.ir)[i] : T(0);
        whp[p] = (MODE == MODE_SYM && own) ? whv[i] : T(0);
        acc[p] = T(0);
    }
    // the symmetric kernel also reaches offsets inside the neighbours' balls
    int reach[RP];
#pragma unroll
    for (int p = 0; p < RP; ++p) {
        const int y = ybase + p;
        reach[p] = (MODE == MODE_SYM) ? ((x < n && y < n) ? a.cnt_thr[x + (int64_t)n * y] : -1)
                                      : thr[p];
        tmax = max(tmax, reach[p]);
    }
    const int rx = min(R, (int)sqrtf((float)max(tmax, 0)) + 1);
    const int col0 = threadIdx.x + R;
    const int row0 = threadIdx.y * RP + R;        // tile row of output p = row0 + p

    // one output's term for the window element v at offset (ox, oy); MASKED checks the
    // horizon, the unmasked core is only entered where every output's ball holds the row
    auto term = [&](int p, const Elem &v, int o2, T g, bool masked) {
        if constexpr (MODE == MODE_SYM) {
            const T wi = (o2 <= thr[p]) ? whp[p] : T(0);
            const T wj = (o2 <= v.thr) ? v.wh : T(0);
            acc[p] += g * v.b * (wi + wj) * (v.u - ui[p]);
        } else if constexpr (MODE == MODE_POLY) {
            if (!masked || o2 <= thr[p])
                acc[p] += poly_weight<T>(a.poly, a.K, (T)o2 * irp[p]) * v.b * (v.u - ui[p]);
        } else {
            if (!masked || o2 <= thr[p]) acc[p] += g * v.b * (v.u - ui[p]);
        }
    };

    for (int ox = -rx; ox <= rx; ++ox) {
        const int ox2 = ox * ox;
        if (ox2 > tmax) continue;
        // per-output half-heights of this column: |oy| <= h_p  <=>  ox^2 + oy^2 <= reach_p
        int hmin = R, hmax = -1;
#pragma unroll
        for (int p = 0; p < RP; ++p) {
            int h = -1;
            const int rest = reach[p] - ox2;
            if (rest >= 0) {
                h = (int)sqrtf((float)rest);
                while (h * h > rest) --h;
                while ((h + 1) * (h + 1) <= rest) ++h;
            }
            hmin = min(hmin, h);
            hmax = max(hmax, h);
        }
        if (hmax < 0) continue;
        hmax = min(hmax, R);
        if (MODE == MODE_SYM) hmin = -1;            // every term carries its own masks
        const Elem *colp = tile + col0 + ox;
        const T *gcol = s_g + (ox + R) * GW + R;
        Elem W[RP];
        int oy = -hmax;
#pragma unroll
        for (int k = 0; k < RP; ++k) W[k] = colp[(row0 + oy + k) * SX];
        // rows where some output's ball ends: single masked steps
        auto single = [&](int oyv) {
            const int o2 = ox2 + oyv * oyv;
            const T g = (MODE == MODE_POLY) ? T(1) : gcol[oyv];
#pragma unroll
            for (int p = 0; p < RP; ++p) term(p, W[p], o2, g, true);
#pragma unroll
            for (int k = 0; k < RP - 1; ++k) W[k] = W[k + 1];
            W[RP - 1] = colp[(row0 + oyv + RP) * SX];
        };
        for (; oy < -hmin && oy <= hmax; ++oy) single(oy);
        // core: every output's ball holds rows -hmin .. hmin; unmasked chunks of RP rows
        for (; oy + RP - 1 <= hmin; oy += RP) {
            Elem X[RP - 1];
#pragma unroll
            for (int k = 0; k < RP - 1; ++k) X[k] = colp[(row0 + oy + RP + k) * SX];
#pragma unroll
            for (int j = 0; j < RP; ++j) {
                const int oyj = oy + j;
                const int o2 = ox2 + oyj * oyj;
                const T g = (MODE == MODE_POLY) ? T(1) : gcol[oyj];
#pragma unroll
                for (int p = 0; p < RP; ++p) {
                    const int k = p + j;
                    term(p, k < RP ? W[k] : X[k - RP], o2, g, false);
                }
            }
#pragma unroll
            for (int k = 0; k < RP - 1; ++k) W[k] = X[k];
            W[RP - 1] = colp[(row0 + oy + 2 * RP - 1) * SX];
        }
        for (; oy <= hmax; ++oy) single(oy);
    }
    const T *__restrict__ finv = (const T *)a.fin;
    const T *__restrict__ extv = (const T *)a.ext;
#pragma unroll
    for (int p = 0; p < RP; ++p) {
        const int y = ybase + p;
        if (x < n && y < n) {
            const int64_t i = x + (int64_t)n * y;
            Lu[(int64_t)blockIdx.z * N + i] = finv[i] * (acc[p] - ui[p] * extv[i]);
        }
    }
}

// ---------------------------------------------------------------------------
// 2-D register-blocked FP32 kernel with paired FP32 arithmetic (POWER kernels).  Same
// traversal as k_direct2d_rb, but each thread owns two adjacent columns of RB_P rows,
// and every multiply/add runs as one paired f32x2 instruction on the two columns (per element
// IEEE round-to-nearest, so each column's result is bitwise the single-column one).  A block of
// 32 x TY threads covers 64 columns and TY * RB_P rows (TY = 2 or 4, chosen per plan by timing
// both); the tile is kept as separate u and b planes so that a warp's pair loads cover 64
// consecutive floats.  A thread's outputs and its summation order do not depend on TY.
// Adjacent columns have close horizons, so few rows of a column offset need per-output masks.
// ---------------------------------------------------------------------------
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t f2_pack(float lo, float hi)
{
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b)
{
    f2_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b)
{
    f2_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b)
{
    f2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c)
{
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// asynchronous 4-byte global -> shared copy (zero-filled when !ok), and the wait for all of a
// thread's outstanding copies
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool ok)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;"
                 ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ int isqrt_small(int x)   // floor(sqrt(x)), 0 <= x < 2^24
{
    int h = (int)sqrtf((float)x);
    h -= (h * h > x);
    h += ((h + 1) * (h + 1) <= x);
    return h;
}

// Row pairs of the tile: lane l owns the adjacent columns 2l and 2l + 1 (two 4-byte loads, as
// the column offset may be odd).
__device__ __forceinline__ f2_t ld_pair(const float *p) { return f2_pack(p[0], p[1]); }

// four consecutive tile rows of the u and b planes at one column offset
struct X2Grp { f2_t u[4], b[4]; };

__device__ __forceinline__ void x2_load_grp(X2Grp &g, const float *cu, int plane, int SX, int row)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        g.u[k] = ld_pair(cu + (row + k) * SX);
        g.b[k] = ld_pair(cu + (row + k) * SX + plane);
    }
}

// Per-output weights of the kappa part of the splitting (Sec. 3) on the paired-column tile,
// K <= 1: w = ra g(o) - p0 - p1 |o|^2 / R2 = fma(ra, g, fma(bk, |o|^2, c0)), ra = R^alpha,
// bk = -p1 / R2 per output (the column pair), c0 = -p0.  KAP = false: w = g (NL_POWER).
struct X2Kap { f2_t ra[RB_P], bk[RB_P], c0; };

template <bool KAP>
__device__ __forceinline__ f2_t x2_w(const X2Kap &kp, int p, f2_t gg, float o2)
{
    if (!KAP) return gg;
    return f2_fma(kp.ra[p], gg, f2_fma(kp.bk[p], f2_pack(o2, o2), kp.c0));
}

// rows oy .. oy + 3 (weights g4) for the RB_P (= 8) outputs; the window is (G0, G1) = rows
// oy .. oy + 7 and G2 holds rows oy + 8 .. oy + 11; every output is inside its ball
template <bool KAP = false>
__device__ __forceinline__ void x2_core4(f2_t (&acc)[RB_P], const f2_t (&ui)[RB_P],
                                         const X2Grp &G0, const X2Grp &G1, const X2Grp &G2,
                                         const float (&g4)[4], const X2Kap &kp, float o2base,
                                         int oy)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float g = g4[j];
        const f2_t gg = f2_pack(g, g);
        const float o2 = KAP ? o2base + (float)((oy + j) * (oy + j)) : 0.f;
#pragma unroll
        for (int p = 0; p < RB_P; ++p) {
            const int k = p + j;
            const X2Grp &G = k < 4 ? G0 : (k < 8 ? G1 : G2);
            acc[p] = f2_fma(f2_mul(G.b[k & 3], x2_w<KAP>(kp, p, gg, o2)),
                            f2_sub(G.u[k & 3], ui[p]), acc[p]);
        }
    }
}

// thresholds of a thread's two output columns (0 off the grid)
struct X2Thr { int a[RB_P], b[RB_P]; };

// one row (offset oy) for the RB_P outputs from the window (G0, G1); MASK: outputs whose ball
// does not hold the offset get weight 0
template <bool MASK, bool KAP = false>
__device__ __forceinline__ void x2_row(f2_t (&acc)[RB_P], const f2_t (&ui)[RB_P],
                                       const X2Grp &G0, const X2Grp &G1,
                                       const X2Thr &thr2, float g, int o2, const X2Kap &kp)
{
#pragma unroll
    for (int p = 0; p < RB_P; ++p) {
        const X2Grp &G = p < 4 ? G0 : G1;
        f2_t gm;
        if (KAP) {
            float wa, wb;
            f2_unpack(x2_w<true>(kp, p, f2_pack(g, g), (float)o2), wa, wb);
            gm = MASK ? f2_pack(o2 <= thr2.a[p] ? wa : 0.f, o2 <= thr2.b[p] ? wb : 0.f)
                      : f2_pack(wa, wb);
        } else {
            gm = MASK ? f2_pack(o2 <= thr2.a[p] ? g : 0.f, o2 <= thr2.b[p] ? g : 0.f)
                      : f2_pack(g, g);
        }
        acc[p] = f2_fma(f2_mul(G.b[p & 3], gm), f2_sub(G.u[p & 3], ui[p]), acc[p]);
    }
}

// slide the window (G0, G1) down one row, loading row `row` + 8 when `more`
__device__ __forceinline__ void x2_slide(X2Grp &G0, X2Grp &G1, const float *cu, int plane,
                                         int SX, int row, bool more)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) { G0.u[k] = G0.u[k + 1]; G0.b[k] = G0.b[k + 1]; }
    G0.u[3] = G1.u[0]; G0.b[3] = G1.b[0];
#pragma unroll
    for (int k = 0; k < 3; ++k) { G1.u[k] = G1.u[k + 1]; G1.b[k] = G1.b[k + 1]; }
    if (more) {
        G1.u[3] = ld_pair(cu + (row + 8) * SX);
        G1.b[3] = ld_pair(cu + (row + 8) * SX + plane);
    }
}

// one column offset ox: rows -hmax .. hmax in increasing order (the same order for every
// output), masked single rows at the rims, unmasked groups of four rows in the core with the
// three row groups rotated instead of copied, and each group's four weights loaded one group
// ahead (indices clamped to the column's last row, so no read leaves the column).  hmin and
// hmax are the same for the whole warp (its 64 x 8 outputs), so every lane runs the same loops.
template <bool KAP = false>
__device__ __forceinline__ void x2_column(f2_t (&acc)[RB_P], const f2_t (&ui)[RB_P],
                                          const X2Thr &thr2, const float *cu, int plane, int SX,
                                          const float *gcol, int ox2, int hmin, int hmax,
                                          const X2Kap &kp)
{
    X2Grp G0, G1, G2;
    int oy = -hmax;
    x2_load_grp(G0, cu, plane, SX, oy);
    x2_load_grp(G1, cu, plane, SX, oy + 4);
    // top rim (or every row when no output's ball covers the centre row of this column)
    const int core_lo = hmin >= 0 ? -hmin : hmax + 1;
    for (; oy < core_lo; ++oy) {
        x2_row<true, KAP>(acc, ui, G0, G1, thr2, gcol[oy], ox2 + oy * oy, kp);
        x2_slide(G0, G1, cu, plane, SX, oy, oy < hmax);
    }
    if (hmin >= 0) {
        int rem = hmin - oy + 1;
        float gc[4], gn[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) gc[j] = gcol[min(oy + j, hmax)];
        auto next_g = [&]() {
#pragma unroll
            for (int j = 0; j < 4; ++j) gn[j] = gcol[min(oy + 4 + j, hmax)];
        };
        auto rotate_g = [&]() {
#pragma unroll
            for (int j = 0; j < 4; ++j) gc[j] = gn[j];
        };
        for (;;) {
            if (rem < 4) break;
            x2_load_grp(G2, cu, plane, SX, oy + 8);
            next_g();
            x2_core4<KAP>(acc, ui, G0, G1, G2, gc, kp, (float)ox2, oy);
            rotate_g();
            oy += 4; rem -= 4;                      // the window is (G1, G2)
            if (rem < 4) { G0 = G1; G1 = G2; break; }
            x2_load_grp(G0, cu, plane, SX, oy + 8);
            next_g();
            x2_core4<KAP>(acc, ui, G1, G2, G0, gc, kp, (float)ox2, oy);
            rotate_g();
            oy += 4; rem -= 4;                      // the window is (G2, G0)
            if (rem < 4) { G1 = G0; G0 = G2; break; }
            x2_load_grp(G1, cu, plane, SX, oy + 8);
            next_g();
            x2_core4<KAP>(acc, ui, G2, G0, G1, gc, kp, (float)ox2, oy);
            rotate_g();
            oy += 4; rem -= 4;                      // the window is (G0, G1) again
        }
        for (; oy <= hmin; ++oy) {
            x2_row<false, KAP>(acc, ui, G0, G1, thr2, gcol[oy], ox2 + oy * oy, kp);
            x2_slide(G0, G1, cu, plane, SX, oy, oy < hmax);
        }
    }
    // bottom rim
    for (; oy <= hmax; ++oy) {
        x2_row<true, KAP>(acc, ui, G0, G1, thr2, gcol[oy], ox2 + oy * oy, kp);
        x2_slide(G0, G1, cu, plane, SX, oy, oy < hmax);
    }
}

// rows oy .. oy + NJ - 1 (NJ <= 4, weights g4) for the RB_P (= 8) outputs, every output
// inside its ball; the window is (G0, G1) = rows oy .. oy + 7 and G2 holds rows oy + 8 ..
// oy + NJ + 6
template <int NJ>
__device__ __forceinline__ void x2_chunk_full(f2_t (&acc)[RB_P], const f2_t (&ui)[RB_P],
                                              const X2Grp &G0, const X2Grp &G1, const X2Grp &G2,
                                              const float (&g4)[4])
{
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const float g = g4[j];
        const f2_t gg = f2_pack(g, g);
#pragma unroll
        for (int p = 0; p < RB_P; ++p) {
            const int k = p + j;
            const X2Grp &G = k < 4 ? G0 : (k < 8 ? G1 : G2);
            acc[p] = f2_fma(f2_mul(G.b[k & 3], gg), f2_sub(G.u[k & 3], ui[p]), acc[p]);
        }
    }
}

// the first NR rows (row .. row + NR - 1) of a group
template <int NR>
__device__ __forceinline__ void x2_load_rows(X2Grp &g, const float *cu, int plane, int SX, int row)
{
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        g.u[k] = ld_pair(cu + (row + k) * SX);
        g.b[k] = ld_pair(cu + (row + k) * SX + plane);
    }
}

// one column offset whose rows -h .. h are inside every output's ball (constant horizon): the
// rows in increasing order in chunks of four, the three row groups rotated, each chunk's
// weights loaded one chunk ahead, then the last 0..3 rows as one short chunk (no per-row
// window shifts).  Tile rows read: -h .. h + 7 (relative to the thread's first output).
__device__ __forceinline__ void x2_column_full(f2_t (&acc)[RB_P], const f2_t (&ui)[RB_P],
                                               const float *cu, int plane, int SX,
                                               const float *gcol, int h)
{
    X2Grp G0, G1, G2;
    int oy = -h, rem = 2 * h + 1;
    x2_load_grp(G0, cu, plane, SX, oy);
    x2_load_grp(G1, cu, plane, SX, oy + 4);
    float gc[4], gn[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) gc[j] = gcol[min(oy + j, h)];
    auto next_g = [&]() {
#pragma unroll
        for (int j = 0; j < 4; ++j) gn[j] = gcol[min(oy + 4 + j, h)];
    };
    auto rotate_g = [&]() {
#pragma unroll
        for (int j = 0; j < 4; ++j) gc[j] = gn[j];
    };
    for (;;) {
        if (rem < 4) break;
        x2_load_grp(G2, cu, plane, SX, oy + 8);
        next_g();
        x2_chunk_full<4>(acc, ui, G0, G1, G2, gc);
        rotate_g();
        oy += 4; rem -= 4;                      // the window is (G1, G2)
        if (rem < 4) { G0 = G1; G1 = G2; break; }
        x2_load_grp(G0, cu, plane, SX, oy + 8);
        next_g();
        x2_chunk_full<4>(acc, ui, G1, G2, G0, gc);
        rotate_g();
        oy += 4; rem -= 4;                      // the window is (G2, G0)
        if (rem < 4) { G1 = G0; G0 = G2; break; }
        x2_load_grp(G1, cu, plane, SX, oy + 8);
        next_g();
        x2_chunk_full<4>(acc, ui, G2, G0, G1, gc);
        rotate_g();
        oy += 4; rem -= 4;                      // the window is (G0, G1) again
    }
    // the last rem rows oy .. h: G2 needs rows oy + 8 .. h + 7 only
    if (rem == 3) {
        x2_load_rows<2>(G2, cu, plane, SX, oy + 8);
        x2_chunk_full<3>(acc, ui, G0, G1, G2, gc);
    } else if (rem == 2) {
        x2_load_rows<1>(G2, cu, plane, SX, oy + 8);
        x2_chunk_full<2>(acc, ui, G0, G1, G2, gc);
    } else if (rem == 1) {
        x2_chunk_full<1>(acc, ui, G0, G1, G2, gc);
    }
}

// RM: compile-time halo (>= the plan's largest radius) so that the tile geometry is constant.
// Persistent: each block takes 64 x (TY * RB_P) tiles (times right-hand sides) from a queue
// ordered by decreasing cost (the sum of the tile's ball sizes, largest first); the last
// block to finish resets the queue for the next launch on the stream.  A block has 2 TY
// warps: warp w takes rows 8 (w / 2) .. 8 (w / 2) + 7 of the tile and the column offsets
// ox even (w even) or odd (w odd), so a tile is half the size of one with a warp per row
// group and the per-item costs even out across the SMs.  The two partial sums of an output
// (each over its column offsets in increasing order) are added once, even part + odd part,
// through shared memory.  The weight table |o|^{-alpha} is copied to shared memory once
// per block.
template <int RM, int TY, int MB, bool KAP = false>
__global__ void __launch_bounds__(64 * TY, MB)
k_direct2d_x2(DirectArgs a, const float *__restrict__ gtab, const float *__restrict__ u,
              float *__restrict__ Lu, const int *__restrict__ order, int ntiles, int tiles_x,
              int nrhs, int *__restrict__ queue)
{
    constexpr int SX = 64 + 2 * RM;                  // even: pair loads stay 8-byte aligned
    constexpr int SY = TY * RB_P + 2 * RM + 1;       // one spare row below the halo
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    const int n = a.n, R = a.R;                      // R <= RM
    float *su = reinterpret_cast<float *>(smem_raw);
    float *sb = su + SX * SY;
    float *sg = sb + SX * SY;                        // [2R+1][2R+1] weights
    f2_t *sx = reinterpret_cast<f2_t *>(smem_raw);   // partial sums, over the tile once read
    const int64_t N = a.N;
    const float *__restrict__ bb = (const float *)a.b;
    const float *__restrict__ finv = (const float *)a.fin;
    const float *__restrict__ extv = (const float *)a.ext;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int grp = threadIdx.y >> 1, half = threadIdx.y & 1;
    const int total = ntiles * nrhs;
    for (int e = tid; e < (2 * R + 1) * (2 * R + 1); e += 64 * TY) sg[e] = gtab[e];
    for (;;) {
        if (tid == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        const int tile = order[item / nrhs], z = item % nrhs;
        const float *__restrict__ ur = u + (int64_t)z * N;
        const int x0 = (tile % tiles_x) * 64, y0 = (tile / tiles_x) * (TY * RB_P);
        // the halo tile by asynchronous 4-byte copies, one warp per tile row and the lanes along
        // x, zero-filled off the grid: every copy of the tile is in flight before the one wait
        for (int row = tid >> 5; row < SY; row += 2 * TY) {
            const int gy = y0 - RM + row;
            const bool rin = gy >= 0 && gy < n;
            const float *__restrict__ urow = ur + (int64_t)n * (rin ? gy : 0);
            const float *__restrict__ brow = bb + (int64_t)n * (rin ? gy : 0);
            for (int xx = tid & 31; xx < SX; xx += 32) {
                const int gx = x0 - RM + xx;
                const bool ok = rin && gx >= 0 && gx < n;
                const int cx = ok ? gx : 0;
                cp_async4(su + row * SX + xx, urow + cx, ok);
                cp_async4(sb + row * SX + xx, brow + cx, ok);
            }
        }
        cp_async_wait_all();
        __syncthreads();

        const int xa = x0 + 2 * threadIdx.x, xb = xa + 1;
        const int ybase = y0 + grp * RB_P;
        f2_t ui[RB_P], acc[RB_P];
        X2Thr thr2;
        X2Kap kp;
        int tmax = -1, tmin = 1 << 30;
        // tile position of output (p = 0, columns xa, xb)
        const float *ua = su + (grp * RB_P + RM) * SX + 2 * threadIdx.x + RM;
        if (KAP) {
            const float p0 = (float)a.poly[0], p1 = a.K >= 1 ? (float)a.poly[1] : 0.f;
            kp.c0 = f2_pack(-p0, -p0);
            const float *__restrict__ whv = (const float *)a.wh;     // R^alpha
            const float *__restrict__ irv = (const float *)a.ir;     // 1 / R2
#pragma unroll
            for (int p = 0; p < RB_P; ++p) {
                const int y = ybase + p;
                const bool oa = xa < n && y < n, ob = xb < n && y < n;
                const int64_t ia = xa + (int64_t)n * y, ib = ia + 1;
                kp.ra[p] = f2_pack(oa ? whv[ia] : 0.f, ob ? whv[ib] : 0.f);
                kp.bk[p] = f2_pack(oa ? -p1 * irv[ia] : 0.f, ob ? -p1 * irv[ib] : 0.f);
            }
        }
#pragma unroll
        for (int p = 0; p < RB_P; ++p) {
            const int y = ybase + p;
            const bool oa = xa < n && y < n, ob = xb < n && y < n;
            const int ta = oa ? a.thr[xa + (int64_t)n * y] : -1;
            const int tb = ob ? a.thr[xb + (int64_t)n * y] : -1;
            thr2.a[p] = max(ta, 0);
            thr2.b[p] = max(tb, 0);
            tmax = max(tmax, max(ta, tb));
            tmin = min(tmin, min(oa ? ta : tmin, ob ? tb : tmin));
            ui[p] = ld_pair(ua + p * SX);
            acc[p] = f2_pack(0.f, 0.f);
        }
        // warp-wide threshold range: every lane takes the same rows of every column offset
        for (int o = 16; o > 0; o >>= 1) {
            tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
            tmin = min(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
        }
        if (tmin == (1 << 30)) tmin = -1;
        const int rx = min(R, isqrt_small(max(tmax, 0)) + 1);
        // the two warps of a row group take the even and the odd column offsets (rows of the
        // two halves within about 1% of each other, where a split by sign differs by the
        // centre column)
        for (int ox = -rx + ((rx + half) & 1); ox <= rx; ox += 2) {
            const int ox2 = ox * ox;
            if (ox2 > tmax) continue;
            const int hmax = min(R, isqrt_small(tmax - ox2));
            const int hmin = (tmin >= ox2) ? min(hmax, isqrt_small(tmin - ox2)) : -1;
            const float *gcol = sg + (ox + R) * (2 * R + 1) + R;       // |oy| <= R
            x2_column<KAP>(acc, ui, thr2, ua + ox, SX * SY, SX, gcol, ox2, hmin, hmax, kp);
        }
        __syncthreads();               // every warp is done with the tile
        f2_t *xs = sx + grp * RB_P * 32 + threadIdx.x;
        if (half) {
#pragma unroll
            for (int p = 0; p < RB_P; ++p) xs[p * 32] = acc[p];
        }
        __syncthreads();
        if (!half) {
#pragma unroll
            for (int p = 0; p < RB_P; ++p) {
                const int y = ybase + p;
                float s0, s1, u0, u1;
                f2_unpack(f2_add(acc[p], xs[p * 32]), s0, s1);
                f2_unpack(ui[p], u0, u1);
                if (y < n && xa < n) {
                    const int64_t i = xa + (int64_t)n * y;
                    Lu[(int64_t)z * N + i] = finv[i] * (s0 - u0 * extv[i]);
                }
                if (y < n && xb < n) {
                    const int64_t i = xb + (int64_t)n * y;
                    Lu[(int64_t)z * N + i] = finv[i] * (s1 - u1 * extv[i]);
                }
            }
        }
        __syncthreads();               // the tile, the partial sums and s_item are reused
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(queue + 1, 1) == (int)gridDim.x - 1) { queue[0] = 0; queue[1] = 0; }
    }
}

template <int RM, int TY>
static size_t x2_smem_bytes()
{
    return sizeof(float) * ((size_t)2 * (64 + 2 * RM) * (TY * RB_P + 2 * RM + 1) +
                            (size_t)(2 * RM + 1) * (2 * RM + 1));
}

// kernel variants: (TY row groups of 8 rows per tile, 2 TY warps per block; minimum resident
// blocks per SM for the register budget)
constexpr int X2_VARIANTS = 4;
static const int x2_var_ty[X2_VARIANTS] = { 1, 1, 2, 2 };

template <int RM, int TY, int MB, bool KAP>
static nl_status launch_x2_t(nl_plan *p, const DirectArgs &a, const float *u, float *Lu,
                             int nrhs, const int *order, int ntiles, int *blocks_cache,
                             cudaStream_t st)
{
    const dim3 blk(32, 2 * TY, 1);
    const size_t smem = x2_smem_bytes<RM, TY>();
    auto kern = k_direct2d_x2<RM, TY, MB, KAP>;
    NL_CUDA_TRY(prep_smem(kern, smem));
    const int tiles_x = (p->n + 63) / 64;
    const int64_t items = (int64_t)ntiles * nrhs;
    if (items >= (int64_t)1 << 31) {
        nl_set_error("nl_apply: %lld tiles x right-hand sides exceed the tile queue", (long long)items);
        return NL_EUNSUPPORTED;
    }
    if (items == 0) return NL_OK;
    if (*blocks_cache == 0) {
        int per_sm = 0, dev = 0, sms = 0;
        NL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 64 * TY, smem));
        NL_CUDA_TRY(cudaGetDevice(&dev));
        NL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        *blocks_cache = (per_sm > 0 ? per_sm : 1) * sms;
    }
    const int64_t blocks = std::min<int64_t>(*blocks_cache, items);
    kern<<<(unsigned)blocks, blk, smem, st>>>(a, p->rb_g32, u, Lu, order, ntiles, tiles_x, nrhs,
                                              p->x2_queue);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

template <int RM, bool KAP>
static nl_status launch_x2_var(nl_plan *p, int var, const DirectArgs &a, const float *u,
                               float *Lu, int nrhs, const int *order, int ntiles, int *bc,
                               cudaStream_t st)
{
    switch (var) {
    case 0: return launch_x2_t<RM, 1, 6, KAP>(p, a, u, Lu, nrhs, order, ntiles, bc, st);
    case 1: return launch_x2_t<RM, 1, 8, KAP>(p, a, u, Lu, nrhs, order, ntiles, bc, st);
    case 2: return launch_x2_t<RM, 2, 3, KAP>(p, a, u, Lu, nrhs, order, ntiles, bc, st);
    default: return launch_x2_t<RM, 2, 4, KAP>(p, a, u, Lu, nrhs, order, ntiles, bc, st);
    }
}

template <bool KAP>
static nl_status x2_launch_any(nl_plan *p, int var, const DirectArgs &a, const float *u,
                               float *Lu, int nrhs, const int *order, int ntiles, int *bc,
                               cudaStream_t st)
{
    if (p->Rmax <= 4) return launch_x2_var<4, KAP>(p, var, a, u, Lu, nrhs, order, ntiles, bc, st);
    if (p->Rmax <= 8) return launch_x2_var<8, KAP>(p, var, a, u, Lu, nrhs, order, ntiles, bc, st);
    if (p->Rmax <= 16) return launch_x2_var<16, KAP>(p, var, a, u, Lu, nrhs, order, ntiles, bc, st);
    if (p->Rmax <= 24) return launch_x2_var<24, KAP>(p, var, a, u, Lu, nrhs, order, ntiles, bc, st);
    return launch_x2_var<32, KAP>(p, var, a, u, Lu, nrhs, order, ntiles, bc, st);
}

// ---------------------------------------------------------------------------
// Symmetric (divergence-form) FP32 kernel with paired columns, on the traversal of
// k_direct2d_x2.  The term of output i and neighbour j at offset o is
//   g(o) b_j (w_i [o^2 <= thr_i] + w_j [o^2 <= thr_j]) (u_j - u_i),
// evaluated as fma(w_i m_i, b_j, c_j m_j) g (u_j - u_i) with c_j = w_j b_j staged per tile and
// the 0/1 masks m = sat(thr + 1 - o^2) (exact: small integers in FP32).  A column offset covers
// the rows up to the warp's largest reach; rows inside the ball of every staged node skip both
// masks, rows inside the ball of every output of the warp skip the output mask.  A mask equal
// to 1 leaves each product bitwise unchanged, so the banding never changes a result.  The tile
// holds four planes: u, b, c and thr + 1 (0 off the grid, where b = c = 0 as well).
// ---------------------------------------------------------------------------
struct X2sGrp { f2_t u[4], b[4], c[4], t[4]; };

// rows row .. row + NR - 1 of the four planes into g (NR < 4 leaves the other entries unset)
template <int NR = 4>
__device__ __forceinline__ void x2s_load_grp(X2sGrp &g, const float *cu, int plane, int SX, int row)
{
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const float *q = cu + (row + k) * SX;
        g.u[k] = ld_pair(q);
        g.b[k] = ld_pair(q + plane);
        g.c[k] = ld_pair(q + 2 * plane);
        g.t[k] = ld_pair(q + 3 * plane);
    }
}

// 0/1 per column of the pair: [o2 <= thr] from t = thr + 1
__device__ __forceinline__ f2_t f2_mask(f2_t t, float o2)
{
    float lo, hi;
    f2_unpack(t, lo, hi);
    return f2_pack(__saturatef(lo - o2), __saturatef(hi - o2));
}

// NJ rows oy .. oy + NJ - 1 for the RB_P outputs; output p at row j reads window entry p + j of
// (A, B, C) = rows oy .. oy + 11.  LVL 0: no masks, 1: node masks, 2: node and output masks.
template <int LVL, int NJ>
__device__ __forceinline__ void x2s_rows(f2_t (&acc)[RB_P], const f2_t (&ui)[RB_P],
                                         const f2_t (&wi)[RB_P], const f2_t (&ti)[RB_P],
                                         const X2sGrp &A, const X2sGrp &B, const X2sGrp &C,
                                         const float *gcol, int oy, float fo)
{
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const float g = gcol[oy + j];
        const f2_t gg = f2_pack(g, g);
        const float o2 = fo + (float)((oy + j) * (oy + j));
#pragma unroll
        for (int p = 0; p < RB_P; ++p) {
            const int k = p + j;
            const X2sGrp &G = k < 4 ? A : (k < 8 ? B : C);
            const f2_t c = LVL >= 1 ? f2_mul(G.c[k & 3], f2_mask(G.t[k & 3], o2)) : G.c[k & 3];
            const f2_t w = LVL >= 2 ? f2_mul(wi[p], f2_mask(ti[p], o2)) : wi[p];
            acc[p] = f2_fma(f2_mul(f2_fma(w, G.b[k & 3], c), gg), f2_sub(G.u[k & 3], ui[p]),
                            acc[p]);
        }
    }
}

// a chunk of four rows at the mask level of its outermost row
__device__ __forceinline__ void x2s_chunk4(f2_t (&acc)[RB_P], const f2_t (&ui)[RB_P],
                                           const f2_t (&wi)[RB_P], const f2_t (&ti)[RB_P],
                                           const X2sGrp &A, const X2sGrp &B, const X2sGrp &C,
                                           const float *gcol, int oy, float fo, int hcore,
                                           int hmid)
{
    const int m = max(abs(oy), abs(oy + 3));
    if (m <= hcore) x2s_rows<0, 4>(acc, ui, wi, ti, A, B, C, gcol, oy, fo);
    else if (m <= hmid) x2s_rows<1, 4>(acc, ui, wi, ti, A, B, C, gcol, oy, fo);
    else x2s_rows<2, 4>(acc, ui, wi, ti, A, B, C, gcol, oy, fo);
}

// the last rem (< 4) rows oy .. oy + rem - 1 = hmax with all masks; (A, B) = rows oy .. oy + 7
// are loaded, C receives rows oy + 8 .. hmax + 7 (the last row any output reads)
__device__ __forceinline__ void x2s_tail(f2_t (&acc)[RB_P], const f2_t (&ui)[RB_P],
                                         const f2_t (&wi)[RB_P], const f2_t (&ti)[RB_P],
                                         const X2sGrp &A, const X2sGrp &B, X2sGrp &C,
                                         const float *cu, int plane, int SX, const float *gcol,
                                         int oy, float fo, int rem)
{
    if (rem == 1) {
        x2s_rows<2, 1>(acc, ui, wi, ti, A, B, C, gcol, oy, fo);
    } else if (rem == 2) {
        x2s_load_grp<1>(C, cu, plane, SX, oy + 8);
        x2s_rows<2, 2>(acc, ui, wi, ti, A, B, C, gcol, oy, fo);
    } else if (rem == 3) {
        x2s_load_grp<2>(C, cu, plane, SX, oy + 8);
        x2s_rows<2, 3>(acc, ui, wi, ti, A, B, C, gcol, oy, fo);
    }
}

// one column offset: rows -hmax .. hmax in increasing order, in chunks of four rows with the
// three register groups rotated (no register shifting), then at most three tail rows.  Band
// limits by |oy|: <= hcore no masks, <= hmid node masks (-1: empty; hcore <= hmid <= hmax).
// hcore, hmid and hmax are the same for the whole warp, so every lane runs the same loops.
__device__ __forceinline__ void x2s_column(f2_t (&acc)[RB_P], const f2_t (&ui)[RB_P],
                                           const f2_t (&wi)[RB_P], const f2_t (&ti)[RB_P],
                                           const float *cu, int plane, int SX, const float *gcol,
                                           int ox2, int hcore, int hmid, int hmax)
{
    X2sGrp G0, G1, G2;
    int oy = -hmax;
    const float fo = (float)ox2;
    x2s_load_grp(G0, cu, plane, SX, oy);
    x2s_load_grp(G1, cu, plane, SX, oy + 4);
    for (;;) {
        if (hmax - oy + 1 < 4) {
            x2s_tail(acc, ui, wi, ti, G0, G1, G2, cu, plane, SX, gcol, oy, fo, hmax - oy + 1);
            break;
        }
        x2s_load_grp(G2, cu, plane, SX, oy + 8);
        x2s_chunk4(acc, ui, wi, ti, G0, G1, G2, gcol, oy, fo, hcore, hmid);
        oy += 4;                                        // the window is (G1, G2)
        if (hmax - oy + 1 < 4) {
            x2s_tail(acc, ui, wi, ti, G1, G2, G0, cu, plane, SX, gcol, oy, fo, hmax - oy + 1);
            break;
        }
        x2s_load_grp(G0, cu, plane, SX, oy + 8);
        x2s_chunk4(acc, ui, wi, ti, G1, G2, G0, gcol, oy, fo, hcore, hmid);
        oy += 4;                                        // the window is (G2, G0)
        if (hmax - oy + 1 < 4) {
            x2s_tail(acc, ui, wi, ti, G2, G0, G1, cu, plane, SX, gcol, oy, fo, hmax - oy + 1);
            break;
        }
        x2s_load_grp(G1, cu, plane, SX, oy + 8);
        x2s_chunk4(acc, ui, wi, ti, G2, G0, G1, gcol, oy, fo, hcore, hmid);
        oy += 4;                                        // the window is (G0, G1) again
    }
}

// Persistent over a largest-first queue of 64 x (TY * RB_P) tiles, with two warps per row group
// splitting the column offsets by parity and adding their partial sums once, as k_direct2d_x2.
template <int RM, int TY, int MB>
__global__ void __launch_bounds__(64 * TY, MB)
k_direct2d_x2s(DirectArgs a, const float *__restrict__ gtab, const float *__restrict__ u,
               float *__restrict__ Lu, const int *__restrict__ order, int ntiles, int tiles_x,
               int nrhs, int *__restrict__ queue)
{
    constexpr int SX = 64 + 2 * RM;
    constexpr int SY = TY * RB_P + 2 * RM + 1;
    constexpr int PL = SX * SY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item, s_jmin[2 * TY];
    const int n = a.n, R = a.R;
    float *su = reinterpret_cast<float *>(smem_raw);          // u | b | c | thr + 1
    const int64_t N = a.N;
    const float *__restrict__ bb = (const float *)a.b;
    const float *__restrict__ whv = (const float *)a.wh;
    const float *__restrict__ finv = (const float *)a.fin;
    const float *__restrict__ extv = (const float *)a.ext;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int grp = threadIdx.y >> 1, half = threadIdx.y & 1;
    f2_t *sx = reinterpret_cast<f2_t *>(smem_raw);           // partial sums, over the tile once read
    const int total = ntiles * nrhs;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        const int tile = order[item / nrhs], z = item % nrhs;
        if (a.skip && a.skip[(int64_t)z * a.skip_stride] != 0.0) {
            __syncthreads();           // every thread has read s_item before it is reused
            continue;
        }
        const float *__restrict__ ur = u + (int64_t)z * N;
        const int x0 = (tile % tiles_x) * 64, y0 = (tile / tiles_x) * (TY * RB_P);
        int jmin = 1 << 30;                          // smallest thr of the staged nodes
        for (int e = tid; e < PL; e += 64 * TY) {
            const int gx = x0 - RM + e % SX, gy = y0 - RM + e / SX;
            float uv = 0.f, bv = 0.f, cv = 0.f, tv = 0.f;
            if (gx >= 0 && gx < n && gy >= 0 && gy < n) {
                const int64_t j = gx + (int64_t)n * gy;
                const int tj = a.thr[j];
                uv = ur[j];
                bv = bb[j];
                cv = whv[j] * bv;
                tv = (float)(tj + 1);
                jmin = min(jmin, tj);
            }
            su[e] = uv;
            su[e + PL] = bv;
            su[e + 2 * PL] = cv;
            su[e + 3 * PL] = tv;
        }
        jmin = __reduce_min_sync(0xffffffffu, jmin);
        if (threadIdx.x == 0) s_jmin[threadIdx.y] = jmin;
        __syncthreads();
#pragma unroll
        for (int w = 0; w < 2 * TY; ++w) jmin = min(jmin, s_jmin[w]);
        const int xa = x0 + 2 * threadIdx.x, xb = xa + 1;
        const int ybase = y0 + grp * RB_P;
        f2_t ui[RB_P], acc[RB_P], wi[RB_P], ti[RB_P];
        int tmax = -1, tmin = 1 << 30;
        const float *ua = su + (grp * RB_P + RM) * SX + 2 * threadIdx.x + RM;
#pragma unroll
        for (int p = 0; p < RB_P; ++p) {
            const int y = ybase + p;
            const bool oa = xa < n && y < n, ob = xb < n && y < n;
            const int64_t ia = xa + (int64_t)n * y, ib = ia + 1;
            const int ta = oa ? a.thr[ia] : -1, tb = ob ? a.thr[ib] : -1;
            const int ra = oa ? a.cnt_thr[ia] : -1, rb = ob ? a.cnt_thr[ib] : -1;
            wi[p] = f2_pack(oa ? whv[ia] : 0.f, ob ? whv[ib] : 0.f);
            ti[p] = f2_pack((float)(ta + 1), (float)(tb + 1));
            tmax = max(tmax, max(ra, rb));
            if (oa) tmin = min(tmin, ta);
            if (ob) tmin = min(tmin, tb);
            ui[p] = ld_pair(ua + p * SX);
            acc[p] = f2_pack(0.f, 0.f);
        }
        tmax = __reduce_max_sync(0xffffffffu, tmax);
        tmin = __reduce_min_sync(0xffffffffu, tmin);
        if (tmin == (1 << 30)) tmin = -1;
        const int cmin = min(tmin, jmin);
        const int rx = min(R, isqrt_small(max(tmax, 0)) + 1);
        // the two warps of a row group take the even and the odd column offsets (rows of the
        // two halves within about 1% of each other, where a split by sign differs by the
        // centre column)
        for (int ox = -rx + ((rx + half) & 1); ox <= rx; ox += 2) {
            const int ox2 = ox * ox;
            if (ox2 > tmax) continue;
            const int hmax = min(R, isqrt_small(tmax - ox2));
            const int hmid = (tmin >= ox2) ? min(hmax, isqrt_small(tmin - ox2)) : -1;
            const int hcore = (cmin >= ox2) ? min(hmid, isqrt_small(cmin - ox2)) : -1;
            const float *gcol = gtab + (ox + R) * (2 * R + 1) + R;     // |oy| <= R
            x2s_column(acc, ui, wi, ti, ua + ox, PL, SX, gcol, ox2, hcore, hmid, hmax);
        }
        __syncthreads();               // every warp is done with the tile
        f2_t *xs = sx + grp * RB_P * 32 + threadIdx.x;
        if (half) {
#pragma unroll
            for (int p = 0; p < RB_P; ++p) xs[p * 32] = acc[p];
        }
        __syncthreads();
        if (!half) {
#pragma unroll
            for (int p = 0; p < RB_P; ++p) {
                const int y = ybase + p;
                float s0, s1, u0, u1;
                f2_unpack(f2_add(acc[p], xs[p * 32]), s0, s1);
                f2_unpack(ui[p], u0, u1);
                if (y < n && xa < n) {
                    const int64_t i = xa + (int64_t)n * y;
                    Lu[(int64_t)z * N + i] = finv[i] * (s0 - u0 * extv[i]);
                }
                if (y < n && xb < n) {
                    const int64_t i = xb + (int64_t)n * y;
                    Lu[(int64_t)z * N + i] = finv[i] * (s1 - u1 * extv[i]);
                }
            }
        }
        __syncthreads();               // the tile, the partial sums, s_item and s_jmin are reused
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(queue + 1, 1) == (int)gridDim.x - 1) { queue[0] = 0; queue[1] = 0; }
    }
}

template <int RM, int TY>
static size_t x2s_smem_bytes()
{
    return sizeof(float) * (size_t)4 * (64 + 2 * RM) * (TY * RB_P + 2 * RM + 1);
}

// symmetric kernel variants: TY warps per tile (shared memory bounds the residency)
constexpr int X2S_VARIANTS = 3;
static const int x2s_var_ty[X2S_VARIANTS] = { 1, 2, 2 };

template <int RM, int TY, int MB>
static nl_status launch_x2s_t(nl_plan *p, const DirectArgs &a, const float *u, float *Lu,
                              int nrhs, const int *order, int ntiles, int *blocks_cache,
                              cudaStream_t st)
{
    const dim3 blk(32, 2 * TY, 1);
    const size_t smem = x2s_smem_bytes<RM, TY>();
    auto kern = k_direct2d_x2s<RM, TY, MB>;
    NL_CUDA_TRY(prep_smem(kern, smem));
    const int tiles_x = (p->n + 63) / 64;
    const int64_t items = (int64_t)ntiles * nrhs;
    if (items >= (int64_t)1 << 31) {
        nl_set_error("nl_apply: %lld tiles x right-hand sides exceed the tile queue", (long long)items);
        return NL_EUNSUPPORTED;
    }
    if (items == 0) return NL_OK;
    if (*blocks_cache == 0) {
        int per_sm = 0, dev = 0, sms = 0;
        NL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 64 * TY, smem));
        NL_CUDA_TRY(cudaGetDevice(&dev));
        NL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        *blocks_cache = (per_sm > 0 ? per_sm : 1) * sms;
    }
    const int64_t blocks = std::min<int64_t>(*blocks_cache, items);
    kern<<<(unsigned)blocks, blk, smem, st>>>(a, p->rb_g32, u, Lu, order, ntiles, tiles_x, nrhs,
                                              p->x2_queue);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

template <int RM>
static nl_status launch_x2s_var(nl_plan *p, int var, const DirectArgs &a, const float *u,
                                float *Lu, int nrhs, const int *order, int ntiles, int *bc,
                                cudaStream_t st)
{
    if (var == 0) return launch_x2s_t<RM, 1, 1>(p, a, u, Lu, nrhs, order, ntiles, bc, st);
    if (var == 1) return launch_x2s_t<RM, 2, 1>(p, a, u, Lu, nrhs, order, ntiles, bc, st);
    return launch_x2s_t<RM, 2, 3>(p, a, u, Lu, nrhs, order, ntiles, bc, st);
}

static nl_status x2s_launch_any(nl_plan *p, int var, const DirectArgs &a, const float *u,
                                float *Lu, int nrhs, const int *order, int ntiles, int *bc,
                                cudaStream_t st)
{
    if (p->Rmax <= 4) return launch_x2s_var<4>(p, var, a, u, Lu, nrhs, order, ntiles, bc, st);
    if (p->Rmax <= 8) return launch_x2s_var<8>(p, var, a, u, Lu, nrhs, order, ntiles, bc, st);
    if (p->Rmax <= 16) return launch_x2s_var<16>(p, var, a, u, Lu, nrhs, order, ntiles, bc, st);
    if (p->Rmax <= 24) return launch_x2s_var<24>(p, var, a, u, Lu, nrhs, order, ntiles, bc, st);
    return launch_x2s_var<32>(p, var, a, u, Lu, nrhs, order, ntiles, bc, st);
}

// ---------------------------------------------------------------------------
// Symmetric FP32 kernel for pairs of right-hand sides (CG applies its operator to all of them at
// once).  Lane l owns one column and RB_P rows, and each paired f32x2 instruction works on the
// two right-hand sides of one output, so the weight of a term,
//   W = (w_i m_i b_j + c_j m_j) g(o),
// and its masks are formed once (scalar FP32) for both.  A warp covers 32 x RB_P outputs (a
// narrower spread of horizons than the 64 x RB_P of k_direct2d_x2s, so fewer masked rows), the
// tile holds (u, u') as one 8-byte plane and b, c, thr + 1 as FP32 planes.  Every output's terms
// are the same FP32 operations in the same order as in k_direct2d_x2s (rows increasing within a
// column offset, column offsets increasing within each parity, the two added once), so each
// right-hand side's result is bit for bit the one k_direct2d_x2s gives for it alone.
// ---------------------------------------------------------------------------
struct X2rGrp { f2_t u[4]; float b[4], c[4], t[4]; };

template <int NR = 4>
__device__ __forceinline__ void x2r_load_grp(X2rGrp &g, const f2_t *cu2, const float *cb, int PL,
                                             int SX, int row)
{
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int o = (row + k) * SX;
        g.u[k] = cu2[o];
        g.b[k] = cb[o];
        g.c[k] = cb[o + PL];
        g.t[k] = cb[o + 2 * PL];
    }
}

// NJ rows oy .. oy + NJ - 1 for the RB_P outputs; output p at row j reads window entry p + j of
// (A, B, C) = rows oy .. oy + 11.  LVL 0: no masks, 1: node masks, 2: node and output masks.
template <int LVL, int NJ>
__device__ __forceinline__ void x2r_rows(f2_t (&acc)[RB_P], const f2_t (&ui)[RB_P],
                                         const float (&wi)[RB_P], const float (&ti)[RB_P],
                                         const X2rGrp &A, const X2rGrp &B, const X2rGrp &C,
                                         const float *gcol, int oy, float fo)
{
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const float g = gcol[oy + j];
        const float o2 = fo + (float)((oy + j) * (oy + j));
#pragma unroll
        for (int p = 0; p < RB_P; ++p) {
            const int k = p + j;
            const X2rGrp &G = k < 4 ? A : (k < 8 ? B : C);
            const float c = LVL >= 1 ? __fmul_rn(G.c[k & 3], __saturatef(G.t[k & 3] - o2))
                                     : G.c[k & 3];
            const float w = LVL >= 2 ? __fmul_rn(wi[p], __saturatef(ti[p] - o2)) : wi[p];
            const float W = __fmul_rn(__fmaf_rn(w, G.b[k & 3], c), g);
            acc[p] = f2_fma(f2_pack(W, W), f2_sub(G.u[k & 3], ui[p]), acc[p]);
        }
    }
}

__device__ __forceinline__ void x2r_chunk4(f2_t (&acc)[RB_P], const f2_t (&ui)[RB_P],
                                           const float (&wi)[RB_P], const float (&ti)[RB_P],
                                           const X2rGrp &A, const X2rGrp &B, const X2rGrp &C,
                                           const float *gcol, int oy, float fo, int hcore,
                                           int hmid)
{
    const int m = max(abs(oy), abs(oy + 3));
    if (m <= hcore) x2r_rows<0, 4>(acc, ui, wi, ti, A, B, C, gcol, oy, fo);
    else if (m <= hmid) x2r_rows<1, 4>(acc, ui, wi, ti, A, B, C, gcol, oy, fo);
    else x2r_rows<2, 4>(acc, ui, wi, ti, A, B, C, gcol, oy, fo);
}

__device__ __forceinline__ void x2r_tail(f2_t (&acc)[RB_P], const f2_t (&ui)[RB_P],
                                         const float (&wi)[RB_P], const float (&ti)[RB_P],
                                         const X2rGrp &A, const X2rGrp &B, X2rGrp &C,
                                         const f2_t *cu2, const float *cb, int PL, int SX,
                                         const float *gcol, int oy, float fo, int rem)
{
    if (rem == 1) {
        x2r_rows<2, 1>(acc, ui, wi, ti, A, B, C, gcol, oy, fo);
    } else if (rem == 2) {
        x2r_load_grp<1>(C, cu2, cb, PL, SX, oy + 8);
        x2r_rows<2, 2>(acc, ui, wi, ti, A, B, C, gcol, oy, fo);
    } else if (rem == 3) {
        x2r_load_grp<2>(C, cu2, cb, PL, SX, oy + 8);
        x2r_rows<2, 3>(acc, ui, wi, ti, A, B, C, gcol, oy, fo);
    }
}

// one column offset: rows -hmax .. hmax in chunks of four with the three groups rotated, then
// at most three tail rows (the band limits of x2s_column)
__device__ __forceinline__ void x2r_column(f2_t (&acc)[RB_P], const f2_t (&ui)[RB_P],
                                           const float (&wi)[RB_P], const float (&ti)[RB_P],
                                           const f2_t *cu2, const float *cb, int PL, int SX,
                                           const float *gcol, int ox2, int hcore, int hmid,
                                           int hmax)
{
    X2rGrp G0, G1, G2;
    int oy = -hmax;
    const float fo = (float)ox2;
    x2r_load_grp(G0, cu2, cb, PL, SX, oy);
    x2r_load_grp(G1, cu2, cb, PL, SX, oy + 4);
    for (;;) {
        if (hmax - oy + 1 < 4) {
            x2r_tail(acc, ui, wi, ti, G0, G1, G2, cu2, cb, PL, SX, gcol, oy, fo, hmax - oy + 1);
            break;
        }
        x2r_load_grp(G2, cu2, cb, PL, SX, oy + 8);
        x2r_chunk4(acc, ui, wi, ti, G0, G1, G2, gcol, oy, fo, hcore, hmid);
        oy += 4;
        if (hmax - oy + 1 < 4) {
            x2r_tail(acc, ui, wi, ti, G1, G2, G0, cu2, cb, PL, SX, gcol, oy, fo, hmax - oy + 1);
            break;
        }
        x2r_load_grp(G0, cu2, cb, PL, SX, oy + 8);
        x2r_chunk4(acc, ui, wi, ti, G1, G2, G0, gcol, oy, fo, hcore, hmid);
        oy += 4;
        if (hmax - oy + 1 < 4) {
            x2r_tail(acc, ui, wi, ti, G2, G0, G1, cu2, cb, PL, SX, gcol, oy, fo, hmax - oy + 1);
            break;
        }
        x2r_load_grp(G1, cu2, cb, PL, SX, oy + 8);
        x2r_chunk4(acc, ui, wi, ti, G2, G0, G1, gcol, oy, fo, hcore, hmid);
        oy += 4;
    }
}

// Persistent over a largest-first queue of (32 x TY RB_P tile, pair of right-hand sides) items;
// two warps per row group split the column offsets by parity (as k_direct2d_x2s).
template <int RM, int TY, int MB>
__global__ void __launch_bounds__(64 * TY, MB)
k_direct2d_x2r(DirectArgs a, const float *__restrict__ gtab, const float *__restrict__ u,
               float *__restrict__ Lu, const int *__restrict__ order, int ntiles, int tiles_x,
               int npairs, int *__restrict__ queue, const float *__restrict__ cpl,
               const float *__restrict__ tpl, const int *__restrict__ tile_jmin)
{
    constexpr int SX = 32 + 2 * RM;
    constexpr int SY = TY * RB_P + 2 * RM + 1;
    constexpr int PL = SX * SY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    f2_t *su2 = reinterpret_cast<f2_t *>(smem_raw);          // (u, u') of the pair
    float *sb = reinterpret_cast<float *>(su2 + PL);         // b | c | thr + 1
    f2_t *sx = su2;                                          // half sums, over the tile once read
    const int n = a.n, R = a.R;
    const int64_t N = a.N;
    const float *__restrict__ bb = (const float *)a.b;
    const float *__restrict__ whv = (const float *)a.wh;
    const float *__restrict__ finv = (const float *)a.fin;
    const float *__restrict__ extv = (const float *)a.ext;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int grp = threadIdx.y >> 1, half = threadIdx.y & 1;
    const int total = ntiles * npairs;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        const int tile = order[item / npairs], z = 2 * (item % npairs);
        if (a.skip && a.skip[(int64_t)z * a.skip_stride] != 0.0 &&
            a.skip[(int64_t)(z + 1) * a.skip_stride] != 0.0) {
            __syncthreads();           // every thread has read s_item before it is reused
            continue;
        }
        const float *__restrict__ u0 = u + (int64_t)z * N;
        const float *__restrict__ u1 = u0 + N;
        const int x0 = (tile % tiles_x) * 32, y0 = (tile / tiles_x) * (TY * RB_P);
        // the tile by asynchronous 4-byte copies (one warp per tile row, zero-filled off the
        // grid): u and u' into the two halves of the pair plane, b, c = (W/2) b and thr + 1 from
        // their plan planes; the smallest threshold of the staged nodes is a plan constant
        for (int row = tid >> 5; row < SY; row += 2 * TY) {
            const int gy = y0 - RM + row;
            const bool rin = gy >= 0 && gy < n;
            const int64_t roff = (int64_t)n * (rin ? gy : 0);
            for (int xx = tid & 31; xx < SX; xx += 32) {
                const int gx = x0 - RM + xx;
                const bool ok = rin && gx >= 0 && gx < n;
                const int64_t j = roff + (ok ? gx : 0);
                const int e = row * SX + xx;
                float *pu = reinterpret_cast<float *>(su2 + e);
                cp_async4(pu, u0 + j, ok);
                cp_async4(pu + 1, u1 + j, ok);
                cp_async4(sb + e, bb + j, ok);
                cp_async4(sb + e + PL, cpl + j, ok);
                cp_async4(sb + e + 2 * PL, tpl + j, ok);
            }
        }
        const int jmin = tile_jmin[tile];
        cp_async_wait_all();
        __syncthreads();
        const int x = x0 + threadIdx.x;
        const int ybase = y0 + grp * RB_P;
        f2_t ui[RB_P], acc[RB_P];
        float wi[RB_P], ti[RB_P];
        int tmax = -1, tmin = 1 << 30;
        const int base = (grp * RB_P + RM) * SX + threadIdx.x + RM;
#pragma unroll
        for (int p = 0; p < RB_P; ++p) {
            const int y = ybase + p;
            const bool o = x < n && y < n;
            const int64_t i = x + (int64_t)n * y;
            const int t = o ? a.thr[i] : -1;
            const int r = o ? a.cnt_thr[i] : -1;
            wi[p] = o ? whv[i] : 0.f;
            ti[p] = (float)(t + 1);
            tmax = max(tmax, r);
            if (o) tmin = min(tmin, t);
            ui[p] = su2[base + p * SX];
            acc[p] = f2_pack(0.f, 0.f);
        }
        tmax = __reduce_max_sync(0xffffffffu, tmax);
        tmin = __reduce_min_sync(0xffffffffu, tmin);
        if (tmin == (1 << 30)) tmin = -1;
        const int cmin = min(tmin, jmin);
        const int rx = min(R, isqrt_small(max(tmax, 0)) + 1);
        // the two warps of a row group take the even and the odd column offsets (rows of the
        // two halves within about 1% of each other, where a split by sign differs by the
        // centre column)
        for (int ox = -rx + ((rx + half) & 1); ox <= rx; ox += 2) {
            const int ox2 = ox * ox;
            if (ox2 > tmax) continue;
            const int hmax = min(R, isqrt_small(tmax - ox2));
            const int hmid = (tmin >= ox2) ? min(hmax, isqrt_small(tmin - ox2)) : -1;
            const int hcore = (cmin >= ox2) ? min(hmid, isqrt_small(cmin - ox2)) : -1;
            const float *gcol = gtab + (ox + R) * (2 * R + 1) + R;     // |oy| <= R
            x2r_column(acc, ui, wi, ti, su2 + base + ox, sb + base + ox, PL, SX, gcol, ox2, hcore,
                       hmid, hmax);
        }
        __syncthreads();               // every warp is done with the tile
        f2_t *xs = sx + grp * RB_P * 32 + threadIdx.x;
        if (half) {
#pragma unroll
            for (int p = 0; p < RB_P; ++p) xs[p * 32] = acc[p];
        }
        __syncthreads();
        if (!half) {
#pragma unroll
            for (int p = 0; p < RB_P; ++p) {
                const int y = ybase + p;
                float s0, s1, v0, v1;
                f2_unpack(f2_add(acc[p], xs[p * 32]), s0, s1);
                f2_unpack(ui[p], v0, v1);
                if (y < n && x < n) {
                    const int64_t i = x + (int64_t)n * y;
                    Lu[(int64_t)z * N + i] = finv[i] * (s0 - v0 * extv[i]);
                    Lu[(int64_t)(z + 1) * N + i] = finv[i] * (s1 - v1 * extv[i]);
                }
            }
        }
        __syncthreads();               // the tile, the half sums, s_item and s_jmin are reused
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(queue + 1, 1) == (int)gridDim.x - 1) { queue[0] = 0; queue[1] = 0; }
    }
}

constexpr int X2R_TY = 2;             // row groups per tile of the pair kernel
constexpr int X2R_MB = 3;             // blocks per SM (168 registers, no spills)

template <int RM>
static size_t x2r_smem_bytes()
{
    return (size_t)(32 + 2 * RM) * (X2R_TY * RB_P + 2 * RM + 1) * (sizeof(f2_t) + 3 * sizeof(float));
}

template <int RM>
static nl_status launch_x2r_t(nl_plan *p, const DirectArgs &a, const float *u, float *Lu,
                              int npairs, cudaStream_t st)
{
    constexpr int TY = X2R_TY;
    const dim3 blk(32, 2 * TY, 1);
    const size_t smem = x2r_smem_bytes<RM>();
    auto kern = k_direct2d_x2r<RM, TY, X2R_MB>;
    NL_CUDA_TRY(prep_smem(kern, smem));
    const int tiles_x = (p->n + 31) / 32;
    const int64_t items = (int64_t)p->x2r_tiles * npairs;
    if (items >= (int64_t)1 << 31) {
        nl_set_error("nl_apply: %lld tiles x right-hand-side pairs exceed the tile queue",
                     (long long)items);
        return NL_EUNSUPPORTED;
    }
    if (items == 0) return NL_OK;
    if (p->x2r_blocks == 0) {
        int per_sm = 0, dev = 0, sms = 0;
        NL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 64 * TY, smem));
        NL_CUDA_TRY(cudaGetDevice(&dev));
        NL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        p->x2r_blocks = (per_sm > 0 ? per_sm : 1) * sms;
    }
    const int64_t blocks = std::min<int64_t>(p->x2r_blocks, items);
    kern<<<(unsigned)blocks, blk, smem, st>>>(a, p->rb_g32, u, Lu, p->x2r_order, p->x2r_tiles,
                                              tiles_x, npairs, p->x2r_queue, p->x2r_c32,
                                              p->x2r_tp1, p->x2r_jmin);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

static nl_status x2r_launch_any(nl_plan *p, const DirectArgs &a, const float *u, float *Lu,
                                int npairs, cudaStream_t st)
{
    if (p->Rmax <= 4) return launch_x2r_t<4>(p, a, u, Lu, npairs, st);
    if (p->Rmax <= 8) return launch_x2r_t<8>(p, a, u, Lu, npairs, st);
    if (p->Rmax <= 16) return launch_x2r_t<16>(p, a, u, Lu, npairs, st);
    if (p->Rmax <= 24) return launch_x2r_t<24>(p, a, u, Lu, npairs, st);
    return launch_x2r_t<32>(p, a, u, Lu, npairs, st);
}

// Plan planes of the pair kernel's tile: c = (W/2) b and thr + 1 per node (the values the tile
// holds, as the kernel used to form them), and per 32 x rows tile the smallest threshold of the
// nodes its halo tile stages (columns x0 - rm .. x0 + 31 + rm, rows y0 - rm .. y0 + rows + rm).
__global__ void k_x2r_planes(int64_t N, const float *__restrict__ wh, const float *__restrict__ b,
                             const int *__restrict__ thr, float *__restrict__ c,
                             float *__restrict__ t)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    c[i] = wh[i] * b[i];
    t[i] = (float)(thr[i] + 1);
}

__global__ void __launch_bounds__(256) k_x2r_tile_jmin(int n, int tiles_x, int rows, int rm,
                                                       const int *__restrict__ thr,
                                                       int *__restrict__ out)
{
    __shared__ int s_w[8];
    const int tile = blockIdx.x;
    const int x0 = (tile % tiles_x) * 32, y0 = (tile / tiles_x) * rows;
    const int sx = 32 + 2 * rm, sy = rows + 2 * rm + 1;
    int m = 1 << 30;
    for (int e = threadIdx.x; e < sx * sy; e += blockDim.x) {
        const int gx = x0 - rm + e % sx, gy = y0 - rm + e / sx;
        if (gx >= 0 && gx < n && gy >= 0 && gy < n) m = min(m, thr[gx + (int64_t)n * gy]);
    }
    m = __reduce_min_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = min(m, s_w[w]);
        out[tile] = m;
    }
}

// Tile order for the paired-column kernel: the cost of a 64 x rows tile is the sum of its
// nodes' ball sizes; tiles are queued largest first.
__global__ void k_x2_tile_cost(int n, int tiles_x, int width, int rows,
                               const int *__restrict__ cnt, long long *__restrict__ cost)
{
    __shared__ long long s_w[8];
    const int tile = blockIdx.x;
    const int x0 = (tile % tiles_x) * width, y0 = (tile / tiles_x) * rows;
    long long c = 0;
    for (int e = threadIdx.x; e < width * rows; e += blockDim.x) {
        const int x = x0 + e % width, y = y0 + e / width;
        if (x < n && y < n) c += cnt[x + (int64_t)n * y];
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) c += s_w[w];
        cost[tile] = c;
    }
}

// largest-first order of the width x (TY * RB_P) tiles, uploaded to *order_dev
static nl_status x2_order_for(nl_plan *p, int ty, int **order_dev, int *ntiles, cudaStream_t st,
                              int width = 64)
{
    const int rows = ty * RB_P;
    const int tiles_x = (p->n + width - 1) / width, tiles_y = (p->n + rows - 1) / rows;
    const int64_t tiles = (int64_t)tiles_x * tiles_y;
    if (tiles >= (int64_t)1 << 30) return NL_EUNSUPPORTED;
    long long *d_cost = nullptr;
    NL_CUDA_TRY(cudaMalloc(&d_cost, tiles * sizeof(long long)));
    std::vector<long long> cost(tiles);
    k_x2_tile_cost<<<(unsigned)tiles, 256, 0, st>>>(p->n, tiles_x, width, rows, p->cnt, d_cost);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cost.data(), d_cost, tiles * sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_cost);
    if (e != cudaSuccess) return nl_cuda_fail(e, "tile costs");
    std::vector<int> order(tiles);
    for (int64_t t = 0; t < tiles; ++t) order[t] = (int)t;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    NL_CUDA_TRY(cudaMalloc(order_dev, tiles * sizeof(int)));
    NL_CUDA_TRY(cudaMemcpyAsync(*order_dev, order.data(), tiles * sizeof(int),
                                cudaMemcpyHostToDevice, st));
    NL_CUDA_TRY(cudaStreamSynchronize(st));
    *ntiles = (int)tiles;
    return NL_OK;
}

// ---------------------------------------------------------------------------
// 3-D FP32 kernel for a constant horizon (POWER kernels): the sum over the ball splits into
// slabs of fixed y offset oy; each slab is the 2-D paired-column sweep above in the x-z plane
// (z the sliding axis, every row inside the common ball, no masks) over the disk of radius^2
// thr - oy^2.  A block of TZ warps covers 64 x 1 x (TZ RB_P) outputs (x, y, z) and stages one
// x-z slab of u and b at a time in shared memory.
// ---------------------------------------------------------------------------
template <int RM, int TZ, int MB>
__global__ void __launch_bounds__(32 * TZ, MB)
k_direct3d_x2(DirectArgs a, const float *__restrict__ g3, const float *__restrict__ u,
              float *__restrict__ Lu, int ztiles)
{
    constexpr int SX = 64 + 2 * RM, SZ = TZ * RB_P + 2 * RM + 1, PL = SX * SZ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *su = reinterpret_cast<float *>(smem_raw);          // u | b
    const int n = a.n, R = a.R;
    const int64_t N = a.N, plane_n = (int64_t)n * n;
    const int rhs = blockIdx.z;
    const float *__restrict__ ur = u + (int64_t)rhs * N;
    const float *__restrict__ bb = (const float *)a.b;
    const int x0 = blockIdx.x * 64;
    const int y = blockIdx.y / ztiles, z0 = (blockIdx.y % ztiles) * (TZ * RB_P);
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int thr = a.thr[0];                                   // the common threshold
    const int xa = x0 + 2 * threadIdx.x, xb = xa + 1;
    const int zbase = z0 + threadIdx.y * RB_P;
    f2_t ui[RB_P], acc[RB_P];
#pragma unroll
    for (int p = 0; p < RB_P; ++p) {
        const int z = zbase + p;
        const float va = (xa < n && z < n) ? ur[xa + n * (y + (int64_t)n * z)] : 0.f;
        const float vb = (xb < n && z < n) ? ur[xb + n * (y + (int64_t)n * z)] : 0.f;
        ui[p] = f2_pack(va, vb);
        acc[p] = f2_pack(0.f, 0.f);
    }
    const int gw = 2 * R + 1;
    const float *ua = su + (threadIdx.y * RB_P + RM) * SX + 2 * threadIdx.x + RM;
    for (int oy = -R; oy <= R; ++oy) {
        const int t2 = thr - oy * oy;
        const int yy = y + oy;
        if (t2 < 0 || yy < 0 || yy >= n) continue;              // slab empty or outside
        __syncthreads();                                         // previous slab consumed
        for (int e = tid; e < PL; e += 32 * TZ) {
            const int gx = x0 - RM + e % SX, gz = z0 - RM + e / SX;
            float uv = 0.f, bv = 0.f;
            if (gx >= 0 && gx < n && gz >= 0 && gz < n) {
                const int64_t j = gx + (int64_t)n * yy + plane_n * gz;
                uv = ur[j];
                bv = bb[j];
            }
            su[e] = uv;
            su[e + PL] = bv;
        }
        __syncthreads();
        const int rx = min(R, isqrt_small(t2));
        for (int ox = -rx; ox <= rx; ++ox) {
            const int ox2 = ox * ox;
            if (ox2 > t2) continue;
            const int h = min(R, isqrt_small(t2 - ox2));
            const float *gcol = g3 + ((oy + R) * gw + (ox + R)) * gw + R;   // oz at gcol[oz]
            x2_column_full(acc, ui, ua + ox, PL, SX, gcol, h);
        }
    }
    const float *__restrict__ finv = (const float *)a.fin;
    const float *__restrict__ extv = (const float *)a.ext;
#pragma unroll
    for (int p = 0; p < RB_P; ++p) {
        const int z = zbase + p;
        if (z >= n) continue;
        float s0, s1, u0, u1;
        f2_unpack(acc[p], s0, s1);
        f2_unpack(ui[p], u0, u1);
        if (xa < n) {
            const int64_t i = xa + n * (y + (int64_t)n * z);
            Lu[(int64_t)rhs * N + i] = finv[i] * (s0 - u0 * extv[i]);
        }
        if (xb < n) {
            const int64_t i = xb + n * (y + (int64_t)n * z);
            Lu[(int64_t)rhs * N + i] = finv[i] * (s1 - u1 * extv[i]);
        }
    }
    (void)tid;
}

// variants (warps per block along z, minimum resident blocks for the register budget),
// timed at plan creation
constexpr int X3_VARIANTS = 4;

template <int RM, int TZ, int MB>
static nl_status launch_3d_x2_t(nl_plan *p, const DirectArgs &a, const float *u, float *Lu,
                                int nrhs, cudaStream_t st)
{
    const size_t smem = sizeof(float) * 2 * (size_t)(64 + 2 * RM) * (TZ * RB_P + 2 * RM + 1);
    auto kern = k_direct3d_x2<RM, TZ, MB>;
    NL_CUDA_TRY(prep_smem(kern, smem));
    const int ztiles = (p->n + TZ * RB_P - 1) / (TZ * RB_P);
    const int64_t gy = (int64_t)p->n * ztiles;
    if (gy > 65535 * 1024LL || nrhs > 65535) {
        nl_set_error("nl_apply: grid too large for the 3-D slab kernel");
        return NL_EUNSUPPORTED;
    }
    const dim3 grd((p->n + 63) / 64, (unsigned)gy, nrhs);
    kern<<<grd, dim3(32, TZ, 1), smem, st>>>(a, p->g3d32, u, Lu, ztiles);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

template <int RM>
static nl_status launch_3d_x2_rm(nl_plan *p, int var, const DirectArgs &a, const float *u,
                                 float *Lu, int nrhs, cudaStream_t st)
{
    switch (var) {
    case 0: return launch_3d_x2_t<RM, 4, 1>(p, a, u, Lu, nrhs, st);
    case 1: return launch_3d_x2_t<RM, 4, 4>(p, a, u, Lu, nrhs, st);
    case 2: return launch_3d_x2_t<RM, 8, 1>(p, a, u, Lu, nrhs, st);
    default: return launch_3d_x2_t<RM, 8, 2>(p, a, u, Lu, nrhs, st);
    }
}

static nl_status launch_3d_x2(nl_plan *p, const DirectArgs &a, const float *u, float *Lu,
                              int nrhs, cudaStream_t st, int var = -1)
{
    if (var < 0) var = p->x3_var;
    if (p->Rmax <= 4) return launch_3d_x2_rm<4>(p, var, a, u, Lu, nrhs, st);
    return launch_3d_x2_rm<8>(p, var, a, u, Lu, nrhs, st);
}

// ---------------------------------------------------------------------------
// Small grids: a group of SPLIT consecutive lanes shares one node; lane g takes the table
// entries g, g + SPLIT, ... of the node's ball (neighbours read through L1), and the group's
// partial sums are combined with shuffles (fixed order).
// ---------------------------------------------------------------------------
template <int D, typename T, int MODE, int SPLIT>
__global__ void __launch_bounds__(256) k_direct_split(DirectArgs a, const T *__restrict__ u,
                                                      T *__restrict__ Lu)
{
    using Entry = typename Tab<T>::type;
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = gid / SPLIT;
    const int lane = (int)(gid % SPLIT);
    const bool own = i < a.N;
    const int n = a.n;
    const int64_t N = a.N;
    const T *__restrict__ ur = u + (int64_t)blockIdx.y * N;
    const T *__restrict__ bb = (const T *)a.b;
    const T *__restrict__ whv = (const T *)a.wh;
    const Entry *__restrict__ tab = (const Entry *)a.tab;
    T acc = T(0), ui = T(0);
    if (own) {
        const int x = (int)(i % n);
        const int y = D > 1 ? (int)((i / n) % n) : 0;
        const int z = D > 2 ? (int)(i / ((int64_t)n * n)) : 0;
        ui = ur[i];
        const int cnt = a.cnt[i];
        const T ir = (MODE == MODE_POLY || MODE == MODE_KAPPA) ? ((const T *)a.ir)[i] : T(0);
        const T whi = (MODE == MODE_SYM || MODE == MODE_KAPPA) ? whv[i] : T(0);
        const int thri = a.thr[i];
        for (int t = lane; t < cnt; t += SPLIT) {
            const int4 o = a.off[t];
            const Entry en = tab[t];
            const int gx = x + o.x, gy = y + o.y, gz = z + o.z;
            if (!in_grid<D>(n, gx, gy, gz)) continue;
            const int64_t j = gx + (int64_t)n * (gy + (int64_t)n * gz);
            const T uj = ur[j], bj = bb[j];
            T w;
            if constexpr (MODE == MODE_POWER) {
                w = (T)en.g * bj;
            } else if constexpr (MODE == MODE_POLY) {
                w = poly_weight<T>(a.poly, a.K, (T)en.o2 * ir) * bj;
            } else if constexpr (MODE == MODE_KAPPA) {
                w = ((T)en.g * whi - poly_weight<T>(a.poly, a.K, (T)en.o2 * ir)) * bj;
            } else {
                const T wi = (en.o2 <= thri) ? whi : T(0);
                const T wj = (en.o2 <= a.thr[j]) ? whv[j] : T(0);
                w = (T)en.g * bj * (wi + wj);
            }
            acc += w * (uj - ui);
        }
    }
#pragma unroll
    for (int o = SPLIT / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, SPLIT);
    if (own && lane == 0) {
        const T fin = ((const T *)a.fin)[i];
        const T ext = ((const T *)a.ext)[i];
        Lu[(int64_t)blockIdx.y * N + i] = fin * (acc - ui * ext);
    }
}

template <int D, typename T, int MODE>
static nl_status launch_split(nl_plan *p, const DirectArgs &a, const T *u, T *Lu, int nrhs,
                              cudaStream_t st)
{
    constexpr int SPLIT = 32;
    const int64_t threads = p->N * SPLIT;
    const dim3 grd((unsigned)((threads + 255) / 256), nrhs, 1);
    k_direct_split<D, T, MODE, SPLIT><<<grd, 256, 0, st>>>(a, u, Lu);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

// ---------------------------------------------------------------------------
// Batched instances in one persistent launch.  Work items are (instance, tile) pairs
// numbered instance by instance; each block takes the next item from an atomic counter,
// stages that instance's halo tile (its own n, R and fields) and applies the instance's
// operator to the tile.  The shared-memory offset of a neighbour is computed from its
// lattice offset, so the tile shape (BX, BY) is free (chosen by the autotuner).
// ---------------------------------------------------------------------------
struct BatchInst {
    DirectArgs a;
    int64_t off;        // element offset of the instance's fields in the concatenated vectors
    int64_t tile0;      // first work item of the instance
    int tiles_x;
};

enum { BK_SCALAR = 0, BK_SYM = 1, BK_PD = 2, BK_PDX2 = 3 };

template <typename T, int KIND, int BX, int BY>
__global__ void __launch_bounds__(BX * BY)
k_batch_persistent(const BatchInst *__restrict__ inst, int ninst, int64_t total,
                   int *__restrict__ counter, const T *__restrict__ u, T *__restrict__ Lu,
                   const double *__restrict__ skip, int skip_stride)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long s_item;
    __shared__ int s_inst;
    const int tid = threadIdx.x + BX * threadIdx.y;
    for (;;) {
        if (tid == 0) {
            const long long it = atomicAdd(counter, 1);
            int k = 0;
            if (it < total) {           // last instance whose first item is <= it
                int hi = ninst - 1;
                while (k < hi) {
                    const int mid = (k + hi + 1) >> 1;
                    if (inst[mid].tile0 <= it) k = mid; else hi = mid - 1;
                }
            }
            s_item = it;
            s_inst = k;
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        if (skip && skip[(size_t)s_inst * skip_stride] != 0.0) {   // instance needs no result
            __syncthreads();
            continue;
        }
        const BatchInst &bi = inst[s_inst];
        const DirectArgs &a = bi.a;
        const int n = a.n, R = a.R;
        const int64_t N = a.N;
        const int64_t local = item - bi.tile0;
        const int x0 = (int)(local % bi.tiles_x) * BX, y0 = (int)(local / bi.tiles_x) * BY;
        const int sx = BX + 2 * R, sy = BY + 2 * R;
        const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
        const bool own = x < n && y < n;
        const int64_t i = own ? x + (int64_t)n * y : 0;
        const int centre = (threadIdx.x + R) + sx * (threadIdx.y + R);
        const T *__restrict__ bb = (const T *)a.b;
        if constexpr (KIND == BK_PD) {
            PdV<T> *tile = reinterpret_cast<PdV<T> *>(smem_raw);
            const T *__restrict__ ux = u + bi.off;
            const T *__restrict__ uy = ux + N;
            for (int e = tid; e < sx * sy; e += BX * BY) {
                const int gx = x0 - R + e % sx, gy = y0 - R + e / sx;
                PdV<T> v;
                if (gx >= 0 && gx < n && gy >= 0 && gy < n) {
                    const int64_t j = gx + (int64_t)n * gy;
                    v.ux = ux[j]; v.uy = uy[j]; v.c = bb[j]; v.in = T(1);
                } else {
                    v.ux = T(0); v.uy = T(0); v.c = T(0); v.in = T(0);
                }
                tile[e] = v;
            }
            __syncthreads();
            if (own) {
                using Entry = typename Tab<T>::pd;
                const Entry *__restrict__ tab = (const Entry *)a.tab;
                const T uxi = ux[i], uyi = uy[i], ci = bb[i];
                const int cnt = a.cnt[i];
                double sxa = 0.0, sya = 0.0;
                T px = T(0), py = T(0);
                for (int t = 0; t < cnt; ++t) {
                    const int4 o = a.off[t];
                    const Entry en = tab[t];
                    const PdV<T> v = tile[centre + o.x + sx * o.y];
                    const T w = ci * v.in + v.c;
                    const T dx = v.ux - uxi, dy = v.uy - uyi;
                    px += w * ((T)en.gxx * dx + (T)en.gxy * dy);
                    py += w * ((T)en.gxy * dx + (T)en.gyy * dy);
                    if ((t & 31) == 31) { sxa += (double)px; sya += (double)py; px = T(0); py = T(0); }
                }
                sxa += (double)px;
                sya += (double)py;
                const double *E = a.pdext + 3 * i;
                const double ox = a.pd_scale * (0.5 * sxa - (E[0] * (double)uxi + E[1] * (double)uyi));
                const double oy = a.pd_scale * (0.5 * sya - (E[1] * (double)uxi + E[2] * (double)uyi));
                T *out = Lu + bi.off;
                out[i] = (T)ox;
                out[N + i] = (T)oy;
            }
        } else {
            using Elem = typename std::conditional<KIND == BK_SYM, V4<T>, V2<T>>::type;
            using Entry = typename Tab<T>::type;
            Elem *tile = reinterpret_cast<Elem *>(smem_raw);
            const T *__restrict__ ur = u + bi.off;
            const T *__restrict__ whv = (const T *)a.wh;
            for (int e = tid; e < sx * sy; e += BX * BY) {
                const int gx = x0 - R + e % sx, gy = y0 - R + e / sx;
                Elem v;
                if (gx >= 0 && gx < n && gy >= 0 && gy < n) {
                    const int64_t j = gx + (int64_t)n * gy;
                    v.u = ur[j];
                    v.b = bb[j];
                    if constexpr (KIND == BK_SYM) { v.wh = whv[j]; v.thr = a.thr[j]; }
                } else {
                    v.u = T(0);
                    v.b = T(0);
                    if constexpr (KIND == BK_SYM) { v.wh = T(0); v.thr = -1; }
                }
                tile[e] = v;
            }
            __syncthreads();
            if (own) {
                const Entry *__restrict__ tab = (const Entry *)a.tab;
                const T ui = ur[i];
                const int cnt = a.cnt[i];
                const T whi = (KIND == BK_SYM) ? whv[i] : T(0);
                const int thri = a.thr[i];
                T acc = T(0);
                for (int t = 0; t < cnt; ++t) {
                    const int4 o = a.off[t];
                    const Entry en = tab[t];
                    const Elem v = tile[centre + o.x + sx * o.y];
                    T w;
                    if constexpr (KIND == BK_SYM) {
                        const T wi = (en.o2 <= thri) ? whi : T(0);
                        const T wj = (en.o2 <= v.thr) ? v.wh : T(0);
                        w = (T)en.g * v.b * (wi + wj);
                    } else {
                        w = (T)en.g * v.b;
                    }
                    acc += w * (v.u - ui);
                }
                const T fin = ((const T *)a.fin)[i];
                const T ext = ((const T *)a.ext)[i];
                Lu[bi.off + i] = fin * (acc - ui * ext);
            }
        }
        __syncthreads();               // the tile and s_item are reused by the next item
    }
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
    // below 32 KB no opt-in is needed even with a kernel's static shared arrays (the
    // default limit covers static + dynamic <= 48 KB)
    if (bytes <= 32 * 1024) return cudaSuccess;
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

template <typename T, int MODE, int RP>
static nl_status launch_rb_tp(nl_plan *p, const DirectArgs &a, const T *u, T *Lu, int nrhs,
                              cudaStream_t st)
{
    const dim3 blk(32, RB_TY, 1);
    const dim3 grd((p->n + 31) / 32, (p->n + RB_TY * RP - 1) / (RB_TY * RP), nrhs);
    const size_t smem = sizeof(T) == 4 ? p->rb_smem32 : p->rb_smem64;   // sized for RB_P >= RP
    const T *g = sizeof(T) == 4 ? (const T *)p->rb_g32 : (const T *)p->rb_g64;
    auto kern = k_direct2d_rb<T, MODE, RP>;
    NL_CUDA_TRY(prep_smem(kern, smem));
    kern<<<grd, blk, smem, st>>>(a, g, u, Lu);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

// Rows per thread: 8 when the grid gives every SM several blocks, else 2.
template <typename T, int MODE>
static nl_status launch_rb_t(nl_plan *p, const DirectArgs &a, const T *u, T *Lu, int nrhs,
                             cudaStream_t st)
{
    const int64_t blocks8 = (int64_t)((p->n + 31) / 32) * ((p->n + RB_TY * RB_P - 1) / (RB_TY * RB_P)) * nrhs;
    if (blocks8 >= 4 * 152) return launch_rb_tp<T, MODE, RB_P>(p, a, u, Lu, nrhs, st);
    return launch_rb_tp<T, MODE, 2>(p, a, u, Lu, nrhs, st);
}

template <typename T>
static nl_status launch_scalar(nl_plan *p, const DirectArgs &a, const T *u, T *Lu, int nrhs,
                               cudaStream_t st, size_t smem)
{
    const int mode = p->symmetric ? MODE_SYM
                   : (p->family == NL_POLY ? MODE_POLY
                      : (p->family == NL_KAPPA ? MODE_KAPPA : MODE_POWER));
    // few nodes with large balls: split each node's ball over a group of lanes
    if (p->N * nrhs < 32 * 1024 && p->num_off >= 64 && nrhs <= 65535) {
#define NL_SPLIT(D)                                                                                \
        do {                                                                                       \
            if (mode == MODE_POWER) return launch_split<D, T, MODE_POWER>(p, a, u, Lu, nrhs, st); \
            if (mode == MODE_POLY) return launch_split<D, T, MODE_POLY>(p, a, u, Lu, nrhs, st);   \
            if (mode == MODE_KAPPA) return launch_split<D, T, MODE_KAPPA>(p, a, u, Lu, nrhs, st); \
            return launch_split<D, T, MODE_SYM>(p, a, u, Lu, nrhs, st);                           \
        } while (0)
        if (p->d == 1) NL_SPLIT(1);
        if (p->d == 2) NL_SPLIT(2);
        NL_SPLIT(3);
#undef NL_SPLIT
    }
    if (p->d == 3 && sizeof(T) == 4 && mode == MODE_POWER && p->g3d32 && p->Rmax <= 8)
        return launch_3d_x2(p, a, (const float *)u, (float *)Lu, nrhs, st);
    if (p->d == 2 && p->rb2d && sizeof(T) == 4 && mode == MODE_KAPPA && p->Rmax <= 32 &&
        p->x2_order)
        return x2_launch_any<true>(p, p->x2_var, a, (const float *)u, (float *)Lu, nrhs,
                                   p->x2_order, p->x2_tiles, &p->x2_blocks, st);
    if (p->d == 2 && p->rb2d && sizeof(T) == 4 && mode != MODE_KAPPA) {
        if (mode == MODE_POWER && p->Rmax <= 32 && p->x2_order) {
            const float *uf = (const float *)u;
            float *lf = (float *)Lu;
            return x2_launch_any<false>(p, p->x2_var, a, uf, lf, nrhs, p->x2_order, p->x2_tiles,
                                        &p->x2_blocks, st);
        }
        if (mode == MODE_SYM && p->Rmax <= 32 && p->x2_order) {
            // pairs of right-hand sides by the pair kernel, an odd last one by x2s (the same
            // bits either way)
            const float *uf = (const float *)u;
            float *lf = (float *)Lu;
            if (nrhs >= 2 && p->x2r_order) {
                nl_status s2 = x2r_launch_any(p, a, uf, lf, nrhs / 2, st);
                if (s2 != NL_OK || nrhs % 2 == 0) return s2;
                const int64_t last = (int64_t)(nrhs - 1) * p->N;
                DirectArgs al = a;             // the last right-hand side is item 0 of this launch
                if (al.skip) al.skip += (int64_t)(nrhs - 1) * al.skip_stride;
                return x2s_launch_any(p, p->x2_var, al, uf + last, lf + last, 1, p->x2_order,
                                      p->x2_tiles, &p->x2_blocks, st);
            }
            return x2s_launch_any(p, p->x2_var, a, uf, lf, nrhs, p->x2_order, p->x2_tiles,
                                  &p->x2_blocks, st);
        }
        if (mode == MODE_POWER) return launch_rb_t<T, MODE_POWER>(p, a, u, Lu, nrhs, st);
        if (mode == MODE_POLY) return launch_rb_t<T, MODE_POLY>(p, a, u, Lu, nrhs, st);
        return launch_rb_t<T, MODE_SYM>(p, a, u, Lu, nrhs, st);
    }
#define NL_DISPATCH_MODE(D)                                                                  \
    do {                                                                                     \
        if (mode == MODE_POWER) return launch_scalar_t<D, T, MODE_POWER>(p, a, u, Lu, nrhs, st, smem); \
        if (mode == MODE_POLY) return launch_scalar_t<D, T, MODE_POLY>(p, a, u, Lu, nrhs, st, smem);   \
        if (mode == MODE_KAPPA) return launch_scalar_t<D, T, MODE_KAPPA>(p, a, u, Lu, nrhs, st, smem); \
        return launch_scalar_t<D, T, MODE_SYM>(p, a, u, Lu, nrhs, st, smem);                 \
    } while (0)
    if (p->d == 1) NL_DISPATCH_MODE(1);
    if (p->d == 2) NL_DISPATCH_MODE(2);
    NL_DISPATCH_MODE(3);
#undef NL_DISPATCH_MODE
}

// ---------------------------------------------------------------------------
// Peridynamic FP32 kernel for a constant horizon, paired columns (as k_direct2d_x2): lane l
// owns the adjacent columns 2l, 2l + 1 of PD_RB rows; a tile is 64 x (TY PD_RB) nodes.  Every
// node has the same ball, so each column offset ox covers rows |oy| <= h(ox) for all outputs
// (exterior neighbours are zero in the tile with in = 0).  Per bond and output pair:
// w = c_i in_j + c_j, d = u_j - u_i, p += w (G d), nine f32x2 instructions.  FP32 partial
// sums over four column offsets at a time (at most 4 (2R+1) bonds) go into FP64 sums.
// ---------------------------------------------------------------------------
constexpr int PD_RB = 4;

struct PdGrp { f2_t ux[4], uy[4], c[4], in[4]; };   // four tile rows of the four planes

__device__ __forceinline__ void pd_load_grp(PdGrp &g, const float *cu, int plane, int SX, int row)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float *r = cu + (row + k) * SX;
        g.ux[k] = ld_pair(r);
        g.uy[k] = ld_pair(r + plane);
        g.c[k] = ld_pair(r + 2 * plane);
        g.in[k] = ld_pair(r + 3 * plane);
    }
}

__device__ __forceinline__ void pd_term(f2_t &px, f2_t &py, f2_t uxi, f2_t uyi, f2_t ci,
                                        f2_t uxj, f2_t uyj, f2_t cj, f2_t inj, f2_t gxx,
                                        f2_t gxy, f2_t gyy)
{
    const f2_t w = f2_fma(ci, inj, cj);
    const f2_t dx = f2_sub(uxj, uxi), dy = f2_sub(uyj, uyi);
    px = f2_fma(w, f2_fma(gxy, dy, f2_mul(gxx, dx)), px);
    py = f2_fma(w, f2_fma(gyy, dy, f2_mul(gxy, dx)), py);
}

// rows oy .. oy + 3 for the PD_RB outputs: window G0 = rows oy .. oy + 3, G1 = the next four
__device__ __forceinline__ void pd_chunk4(f2_t (&px)[PD_RB], f2_t (&py)[PD_RB],
                                          const f2_t (&uxi)[PD_RB], const f2_t (&uyi)[PD_RB],
                                          const f2_t (&ci)[PD_RB], const PdGrp &G0,
                                          const PdGrp &G1, const float *gcol, int oy)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float *g = gcol + 3 * (oy + j);
        const f2_t gxx = f2_pack(g[0], g[0]), gxy = f2_pack(g[1], g[1]), gyy = f2_pack(g[2], g[2]);
#pragma unroll
        for (int p = 0; p < PD_RB; ++p) {
            const int k = p + j;
            const PdGrp &G = k < 4 ? G0 : G1;
            pd_term(px[p], py[p], uxi[p], uyi[p], ci[p], G.ux[k & 3], G.uy[k & 3], G.c[k & 3],
                    G.in[k & 3], gxx, gxy, gyy);
        }
    }
}

__device__ __forceinline__ void pd_flush(f2_t (&px)[PD_RB], f2_t (&py)[PD_RB],
                                         double (&sxa)[PD_RB], double (&sxb)[PD_RB],
                                         double (&sya)[PD_RB], double (&syb)[PD_RB])
{
#pragma unroll
    for (int p = 0; p < PD_RB; ++p) {
        float a0, a1, b0, b1;
        f2_unpack(px[p], a0, a1);
        f2_unpack(py[p], b0, b1);
        sxa[p] += (double)a0; sxb[p] += (double)a1;
        sya[p] += (double)b0; syb[p] += (double)b1;
        px[p] = f2_pack(0.f, 0.f);
        py[p] = px[p];
    }
}

// one 64 x (TY PD_RB) tile whose halo is staged at `sm` (four planes ux, uy, c, in of
// SX x SY); writes both components of every output of the tile
template <int RM, int TY>
__device__ __forceinline__ void pd_x2_tile(const DirectArgs &a, const float *sm, int x0, int y0,
                                           const float *__restrict__ ux,
                                           const float *__restrict__ uy,
                                           float *__restrict__ outx, float *__restrict__ outy)
{
    constexpr int SX = 64 + 2 * RM, SY = TY * PD_RB + 2 * RM + 1, PL = SX * SY;
    const int n = a.n, R = a.R;
    const int xa = x0 + 2 * threadIdx.x, xb = xa + 1;
    const int ybase = y0 + threadIdx.y * PD_RB;
    const float *ua = sm + (threadIdx.y * PD_RB + RM) * SX + 2 * threadIdx.x + RM;
    f2_t uxi[PD_RB], uyi[PD_RB], ci[PD_RB], px[PD_RB], py[PD_RB];
    double sxa[PD_RB], sxb[PD_RB], sya[PD_RB], syb[PD_RB];
#pragma unroll
    for (int p = 0; p < PD_RB; ++p) {
        uxi[p] = ld_pair(ua + p * SX);
        uyi[p] = ld_pair(ua + p * SX + PL);
        ci[p] = ld_pair(ua + p * SX + 2 * PL);
        px[p] = f2_pack(0.f, 0.f);
        py[p] = px[p];
        sxa[p] = sxb[p] = sya[p] = syb[p] = 0.0;
    }
    const int thr = a.thr[0];                        // the common threshold
    const int gw = 2 * R + 1;
    int cols = 0;
    for (int ox = -R; ox <= R; ++ox) {
        const int ox2 = ox * ox;
        if (ox2 > thr) continue;
        const int h = min(R, isqrt_small(thr - ox2));
        const float *gcol = a.pdg + 3 * ((ox + R) * gw + R);    // row oy at gcol[3 oy]
        const float *cu = ua + ox;
        PdGrp G0, G1;
        int oy = -h, rem = 2 * h + 1;
        pd_load_grp(G0, cu, PL, SX, oy);
        for (;;) {
            if (rem < 4) break;
            pd_load_grp(G1, cu, PL, SX, oy + 4);
            pd_chunk4(px, py, uxi, uyi, ci, G0, G1, gcol, oy);
            oy += 4; rem -= 4;                       // the window is G1
            if (rem < 4) { G0 = G1; break; }
            pd_load_grp(G0, cu, PL, SX, oy + 4);
            pd_chunk4(px, py, uxi, uyi, ci, G1, G0, gcol, oy);
            oy += 4; rem -= 4;                       // the window is G0 again
        }
        for (; rem > 0; --rem, ++oy) {
            const float *g = gcol + 3 * oy;
            const f2_t gxx = f2_pack(g[0], g[0]), gxy = f2_pack(g[1], g[1]),
                       gyy = f2_pack(g[2], g[2]);
#pragma unroll
            for (int p = 0; p < PD_RB; ++p)
                pd_term(px[p], py[p], uxi[p], uyi[p], ci[p], G0.ux[p], G0.uy[p], G0.c[p],
                        G0.in[p], gxx, gxy, gyy);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                G0.ux[k] = G0.ux[k + 1]; G0.uy[k] = G0.uy[k + 1];
                G0.c[k] = G0.c[k + 1]; G0.in[k] = G0.in[k + 1];
            }
            if (rem > 1) {
                const float *r = cu + (oy + 4) * SX;
                G0.ux[3] = ld_pair(r); G0.uy[3] = ld_pair(r + PL);
                G0.c[3] = ld_pair(r + 2 * PL); G0.in[3] = ld_pair(r + 3 * PL);
            }
        }
        if (++cols == 4) {                           // FP32 partials into the FP64 sums
            cols = 0;
            pd_flush(px, py, sxa, sxb, sya, syb);
        }
    }
    pd_flush(px, py, sxa, sxb, sya, syb);
#pragma unroll
    for (int p = 0; p < PD_RB; ++p) {
        const int y = ybase + p;
        if (y >= n) continue;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int x = c ? xb : xa;
            if (x >= n) continue;
            const int64_t i = x + (int64_t)n * y;
            const double *E = a.pdext + 3 * i;
            const double uxv = (double)ux[i], uyv = (double)uy[i];
            const double sx = c ? sxb[p] : sxa[p], sy = c ? syb[p] : sya[p];
            outx[i] = (float)(a.pd_scale * (0.5 * sx - (E[0] * uxv + E[1] * uyv)));
            outy[i] = (float)(a.pd_scale * (0.5 * sy - (E[1] * uxv + E[2] * uyv)));
        }
    }
}

// stage the 64 x (TY PD_RB) tile at (x0, y0) with its halo: planes ux, uy, c, in
template <int RM, int TY>
__device__ __forceinline__ void pd_x2_stage(const DirectArgs &a, float *sm, int x0, int y0,
                                            const float *__restrict__ ux,
                                            const float *__restrict__ uy)
{
    constexpr int SX = 64 + 2 * RM, SY = TY * PD_RB + 2 * RM + 1, PL = SX * SY;
    const int n = a.n;
    const float *__restrict__ cc = (const float *)a.b;
    // asynchronous 4-byte copies (one warp per tile row, zero-filled off the grid) for u and c;
    // the inside indicator is a plain store; the caller's barrier follows the wait
    for (int row = threadIdx.y; row < SY; row += TY) {
        const int gy = y0 - RM + row;
        const bool rin = gy >= 0 && gy < n;
        const int64_t roff = (int64_t)n * (rin ? gy : 0);
        for (int xx = threadIdx.x; xx < SX; xx += 32) {
            const int gx = x0 - RM + xx;
            const bool ok = rin && gx >= 0 && gx < n;
            const int64_t j = roff + (ok ? gx : 0);
            const int e = row * SX + xx;
            cp_async4(sm + e, ux + j, ok);
            cp_async4(sm + e + PL, uy + j, ok);
            cp_async4(sm + e + 2 * PL, cc + j, ok);
            sm[e + 3 * PL] = ok ? 1.f : 0.f;
        }
    }
    cp_async_wait_all();
}

template <int RM, int TY>
__global__ void __launch_bounds__(32 * TY)
k_direct_pd_x2(DirectArgs a, const float *__restrict__ u, float *__restrict__ Lu)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sm = reinterpret_cast<float *>(smem_raw);
    const int64_t N = a.N;
    const float *ux = u + (int64_t)blockIdx.z * 2 * N, *uy = ux + N;
    float *ox = Lu + (int64_t)blockIdx.z * 2 * N, *oy = ox + N;
    const int x0 = blockIdx.x * 64, y0 = blockIdx.y * (TY * PD_RB);
    pd_x2_stage<RM, TY>(a, sm, x0, y0, ux, uy);
    __syncthreads();
    pd_x2_tile<RM, TY>(a, sm, x0, y0, ux, uy, ox, oy);
}

template <int RM, int TY>
static size_t pd_x2_smem()
{
    return sizeof(float) * 4 * (size_t)(64 + 2 * RM) * (TY * PD_RB + 2 * RM + 1);
}

template <int RM>
static nl_status launch_pd_x2_rm(nl_plan *p, const DirectArgs &a, const float *u, float *Lu,
                                 int nrhs, cudaStream_t st)
{
    constexpr int TY = 2;
    const size_t smem = pd_x2_smem<RM, TY>();
    auto kern = k_direct_pd_x2<RM, TY>;
    NL_CUDA_TRY(prep_smem(kern, smem));
    const dim3 grd((p->n + 63) / 64, (p->n + TY * PD_RB - 1) / (TY * PD_RB), nrhs);
    kern<<<grd, dim3(32, TY, 1), smem, st>>>(a, u, Lu);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

static nl_status launch_pd_x2(nl_plan *p, const DirectArgs &a, const float *u, float *Lu,
                              int nrhs, cudaStream_t st)
{
    if (p->Rmax <= 4) return launch_pd_x2_rm<4>(p, a, u, Lu, nrhs, st);
    if (p->Rmax <= 8) return launch_pd_x2_rm<8>(p, a, u, Lu, nrhs, st);
    if (p->Rmax <= 16) return launch_pd_x2_rm<16>(p, a, u, Lu, nrhs, st);
    return launch_pd_x2_rm<32>(p, a, u, Lu, nrhs, st);
}

// Batched peridynamic instances (constant horizons, FP32): the persistent (instance, tile)
// queue of k_batch_persistent with the paired-column tile above; tiles are 64 x (TY PD_RB).
template <int RM, int TY>
__global__ void __launch_bounds__(32 * TY)
k_batch_pdx2(const BatchInst *__restrict__ inst, int ninst, int64_t total,
             int *__restrict__ counter, const float *__restrict__ u, float *__restrict__ Lu,
             const double *__restrict__ skip, int skip_stride)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long s_item;
    __shared__ int s_inst;
    float *sm = reinterpret_cast<float *>(smem_raw);
    const int tid = threadIdx.x + 32 * threadIdx.y;
    for (;;) {
        if (tid == 0) {
            const long long it = atomicAdd(counter, 1);
            int k = 0;
            if (it < total) {
                int hi = ninst - 1;
                while (k < hi) {
                    const int mid = (k + hi + 1) >> 1;
                    if (inst[mid].tile0 <= it) k = mid; else hi = mid - 1;
                }
            }
            s_item = it;
            s_inst = k;
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        if (skip && skip[(size_t)s_inst * skip_stride] != 0.0) {   // instance needs no result
            __syncthreads();
            continue;
        }
        const BatchInst &bi = inst[s_inst];
        const int64_t local = item - bi.tile0;
        const int x0 = (int)(local % bi.tiles_x) * 64, y0 = (int)(local / bi.tiles_x) * (TY * PD_RB);
        const float *ux = u + bi.off, *uy = ux + bi.a.N;
        float *ox = Lu + bi.off, *oy = ox + bi.a.N;
        pd_x2_stage<RM, TY>(bi.a, sm, x0, y0, ux, uy);
        __syncthreads();
        pd_x2_tile<RM, TY>(bi.a, sm, x0, y0, ux, uy, ox, oy);
        __syncthreads();               // the tile and s_item are reused by the next item
    }
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
    a.cnt = p->cnt; a.thr = p->thr; a.cnt_thr = p->thr_reach;
    const bool f32 = dtype == NL_F32;
    a.b = f32 ? (const void *)p->b32 : (const void *)p->b64;
    a.fin = f32 ? (const void *)p->fin32 : (const void *)p->fin64;
    a.ext = f32 ? (const void *)p->ext32 : (const void *)p->ext64;
    a.wh = f32 ? (const void *)p->wh32 : (const void *)p->wh64;
    a.ir = f32 ? (const void *)p->ir32 : (const void *)p->ir64;
    a.pdg = p->pd_dense32;
    if (p->family == NL_PD_BOND)
        a.tab = f32 ? (const void *)p->pd32 : (const void *)p->pd64;
    else
        a.tab = f32 ? (const void *)p->tab32 : (const void *)p->tab64;
    a.off = p->off;
    for (int m = 0; m < 8; ++m) a.poly[m] = p->poly[m];
    a.pd_scale = p->sigma * pow(p->h, p->d - 1.0);
    a.pdext = p->pdext;
    a.skip = p->skip_flags;
    a.skip_stride = p->skip_stride;
    return a;
}

nl_status nl_direct_launch(nl_plan *p, const void *u, void *Lu, int nrhs, int dtype,
                           cudaStream_t st)
{
    if (p->family == NL_PD_BOND && p->d != 2) {
        nl_set_error("nl_apply: the direct peridynamic operator is built for d = 2 (a 3-D "
                     "NL_PD_BOND plan serves nl_apply_fast)");
        return NL_EUNSUPPORTED;
    }
    const DirectArgs a = make_args(p, dtype);
    if (p->family == NL_PD_BOND) {
        if (dtype == NL_F32 && p->pd_dense32 && p->Rmax <= 32)
            return launch_pd_x2(p, a, (const float *)u, (float *)Lu, nrhs, st);
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
    if (!u || !Lu || nrhs < 1 || nrhs > 65535 ||
        (dtype != NL_F32 && dtype != NL_F64 && dtype != NL_F64_PAIRS)) {
        nl_set_error("nl_apply: need non-null u/Lu, 1 <= nrhs <= 65535, dtype F32/F64/F64_PAIRS");
        return NL_EINVAL;
    }
    if (p->sym_fast) {
        nl_set_error("nl_apply: the symmetrised NL_POLY operator is applied by nl_apply_fast");
        return NL_EUNSUPPORTED;
    }
    if (dtype == NL_F64_PAIRS)
        return nl_pairs_launch(p, (const double *)u, (double *)Lu, nrhs, nl_stream(stream));
    return nl_direct_launch(p, u, Lu, nrhs, dtype, nl_stream(stream));
}

// ---------------------------------------------------------------------------
// batch launcher (used by nl_batch.cu)
// ---------------------------------------------------------------------------
nl_status nl_batch_fill_inst(nl_plan *const *plans, int count, const int64_t *offsets, int shape,
                             int dtype, int kind, void *host_out, int64_t *total_out)
{
    // generic kernels: 32 x {4, 8, 16} nodes; paired-column PD: 64 x {1, 2, 4} PD_RB nodes
    static const int bxs[3] = { 32, 32, 32 }, bys[3] = { 4, 8, 16 };
    static const int pys[3] = { PD_RB, 2 * PD_RB, 4 * PD_RB };
    const int bx = kind == BK_PDX2 ? 64 : bxs[shape];
    const int by = kind == BK_PDX2 ? pys[shape] : bys[shape];
    BatchInst *bi = reinterpret_cast<BatchInst *>(host_out);
    int64_t t = 0;
    for (int k = 0; k < count; ++k) {
        bi[k].a = make_args(plans[k], dtype);
        bi[k].off = offsets[k];
        bi[k].tile0 = t;
        bi[k].tiles_x = (plans[k]->n + bx - 1) / bx;
        t += (int64_t)bi[k].tiles_x * ((plans[k]->n + by - 1) / by);
    }
    *total_out = t;
    return NL_OK;
}

size_t nl_batch_inst_bytes() { return sizeof(BatchInst); }

template <typename T, int KIND, int BX, int BY>
static nl_status launch_batch_t(const void *inst, int ninst, int64_t total, int *counter,
                                const T *u, T *Lu, int Rmax, cudaStream_t st,
                                const double *skip, int skip_stride)
{
    size_t elem;
    if (KIND == BK_PD) elem = sizeof(PdV<T>);
    else if (KIND == BK_SYM) elem = sizeof(V4<T>);
    else elem = sizeof(V2<T>);
    const size_t smem = elem * (size_t)(BX + 2 * Rmax) * (BY + 2 * Rmax);
    if (smem > 200 * 1024) {
        nl_set_error("batched apply: halo tile of %zu bytes exceeds shared memory", smem);
        return NL_EUNSUPPORTED;
    }
    auto kern = k_batch_persistent<T, KIND, BX, BY>;
    NL_CUDA_TRY(prep_smem(kern, smem));
    int per_sm = 0;
    NL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BX * BY, smem));
    int dev = 0, sms = 0;
    NL_CUDA_TRY(cudaGetDevice(&dev));
    NL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t blocks = (int64_t)(per_sm > 0 ? per_sm : 1) * sms;
    if (blocks > total) blocks = total;
    if (blocks < 1) blocks = 1;
    NL_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), st));
    kern<<<(unsigned)blocks, dim3(BX, BY), smem, st>>>((const BatchInst *)inst, ninst, total,
                                                       counter, u, Lu, skip, skip_stride);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

template <int RM, int TY>
static nl_status launch_batch_pdx2_t(const void *inst, int ninst, int64_t total, int *counter,
                                     const float *u, float *Lu, const double *skip,
                                     int skip_stride, cudaStream_t st)
{
    const size_t smem = pd_x2_smem<RM, TY>();
    auto kern = k_batch_pdx2<RM, TY>;
    NL_CUDA_TRY(prep_smem(kern, smem));
    int per_sm = 0, dev = 0, sms = 0;
    NL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * TY, smem));
    NL_CUDA_TRY(cudaGetDevice(&dev));
    NL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t blocks = (int64_t)(per_sm > 0 ? per_sm : 1) * sms;
    if (blocks > total) blocks = total;
    if (blocks < 1) blocks = 1;
    NL_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), st));
    kern<<<(unsigned)blocks, dim3(32, TY), smem, st>>>((const BatchInst *)inst, ninst, total,
                                                     counter, u, Lu, skip, skip_stride);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

template <int RM>
static nl_status launch_batch_pdx2_rm(int shape, const void *inst, int ninst, int64_t total,
                                      int *counter, const float *u, float *Lu,
                                      const double *skip, int ss, cudaStream_t st)
{
    if (shape == 0) return launch_batch_pdx2_t<RM, 1>(inst, ninst, total, counter, u, Lu, skip, ss, st);
    if (shape == 1) return launch_batch_pdx2_t<RM, 2>(inst, ninst, total, counter, u, Lu, skip, ss, st);
    return launch_batch_pdx2_t<RM, 4>(inst, ninst, total, counter, u, Lu, skip, ss, st);
}

nl_status nl_batch_launch(int kind, int shape, int dtype, const void *inst_dev, int ninst,
                          int64_t total, int *counter, const void *u, void *Lu, int Rmax,
                          cudaStream_t st, const double *skip, int skip_stride)
{
    if (kind == BK_PDX2) {
        if (dtype != NL_F32 || Rmax > 32) {
            nl_set_error("batched apply: paired-column PD needs FP32 and radius <= 32");
            return NL_EINVAL;
        }
        const float *uf = (const float *)u;
        float *lf = (float *)Lu;
        if (Rmax <= 4) return launch_batch_pdx2_rm<4>(shape, inst_dev, ninst, total, counter, uf, lf, skip, skip_stride, st);
        if (Rmax <= 8) return launch_batch_pdx2_rm<8>(shape, inst_dev, ninst, total, counter, uf, lf, skip, skip_stride, st);
        if (Rmax <= 16) return launch_batch_pdx2_rm<16>(shape, inst_dev, ninst, total, counter, uf, lf, skip, skip_stride, st);
        return launch_batch_pdx2_rm<32>(shape, inst_dev, ninst, total, counter, uf, lf, skip, skip_stride, st);
    }
#define NL_BATCH_SHAPES(T, KIND)                                                                   \
    do {                                                                                           \
        if (shape == 0) return launch_batch_t<T, KIND, 32, 4>(inst_dev, ninst, total, counter,    \
                                                              (const T *)u, (T *)Lu, Rmax, st, skip, skip_stride); \
        if (shape == 1) return launch_batch_t<T, KIND, 32, 8>(inst_dev, ninst, total, counter,    \
                                                              (const T *)u, (T *)Lu, Rmax, st, skip, skip_stride); \
        return launch_batch_t<T, KIND, 32, 16>(inst_dev, ninst, total, counter, (const T *)u,     \
                                               (T *)Lu, Rmax, st, skip, skip_stride);              \
    } while (0)
    if (dtype == NL_F32) {
        if (kind == BK_PD) NL_BATCH_SHAPES(float, BK_PD);
        if (kind == BK_SYM) NL_BATCH_SHAPES(float, BK_SYM);
        NL_BATCH_SHAPES(float, BK_SCALAR);
    }
    if (kind == BK_PD) NL_BATCH_SHAPES(double, BK_PD);
    if (kind == BK_SYM) NL_BATCH_SHAPES(double, BK_SYM);
    NL_BATCH_SHAPES(double, BK_SCALAR);
#undef NL_BATCH_SHAPES
}

// ---------------------------------------------------------------------------
// plan-time variant timing: TUNE_ROUNDS rounds over all variants (one untimed launch, then
// TUNE_REPS timed back to back); a variant's time is its fastest round, so one slow round
// (another process on the GPU, a clock change) does not decide the choice.  run(v) launches
// variant v once; ms[v] receives its time.
// ---------------------------------------------------------------------------
constexpr int TUNE_ROUNDS = 3, TUNE_REPS = 3;

template <typename Run>
static nl_status time_variants(int nvar, Run run, float *ms, cudaEvent_t e0, cudaEvent_t e1,
                               cudaStream_t st)
{
    for (int v = 0; v < nvar; ++v) ms[v] = 3.0e38f;
    for (int r = 0; r < TUNE_ROUNDS; ++r) {
        for (int v = 0; v < nvar; ++v) {
            nl_status s = run(v);
            if (s != NL_OK) return s;
            NL_CUDA_TRY(cudaEventRecord(e0, st));
            for (int k = 0; k < TUNE_REPS; ++k)
                if ((s = run(v)) != NL_OK) return s;
            NL_CUDA_TRY(cudaEventRecord(e1, st));
            NL_CUDA_TRY(cudaEventSynchronize(e1));
            float t = 0.f;
            NL_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
            ms[v] = fminf(ms[v], t);
        }
    }
    return NL_OK;
}

// ---------------------------------------------------------------------------
// plan-time set-up of the paired-column FP32 kernel: the tile queue and its orders, and the
// kernel variant (tile height and register budget) chosen by timing each on the plan itself
// ---------------------------------------------------------------------------
static nl_status x3_tune(nl_plan *p, cudaStream_t st)
{
    p->x3_var = 0;
    if (!(p->d == 3 && p->g3d32 && p->Rmax <= 8) || p->N > ((int64_t)1 << 24)) return NL_OK;
    const DirectArgs a = make_args(p, NL_F32);
    float *u = nullptr, *lu = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    nl_status s = NL_OK;
    if (cudaMalloc(&u, p->N * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&lu, p->N * sizeof(float)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMemsetAsync(u, 0, p->N * sizeof(float), st) != cudaSuccess)
        s = nl_cuda_fail(cudaErrorMemoryAllocation, "3-D kernel tuning");
    float ms[X3_VARIANTS];
    if (s == NL_OK)
        s = time_variants(X3_VARIANTS, [&](int v) { return launch_3d_x2(p, a, u, lu, 1, st, v); },
                          ms, e0, e1, st);
    if (s == NL_OK)
        for (int v = 1; v < X3_VARIANTS; ++v) if (ms[v] < ms[p->x3_var]) p->x3_var = v;
    if (u) cudaFree(u);
    if (lu) cudaFree(lu);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return s;
}

nl_status nl_direct_plan_init(nl_plan *p, cudaStream_t st)
{
    if (p->d == 3) return x3_tune(p, st);
    const bool kap = p->family == NL_KAPPA && p->K <= 1;
    if (!(p->d == 2 && p->rb2d && (p->family == NL_POWER || kap) && p->Rmax <= 32)) return NL_OK;
    const bool sym = p->symmetric != 0;
    const int nvar = sym ? X2S_VARIANTS : X2_VARIANTS;
    const int *var_ty = sym ? x2s_var_ty : x2_var_ty;
    NL_CUDA_TRY(cudaMalloc(&p->x2_queue, 2 * sizeof(int)));
    NL_CUDA_TRY(cudaMemsetAsync(p->x2_queue, 0, 2 * sizeof(int), st));
    // tile heights (row groups of 8) of the two kinds of variant: 1 and 2 row groups for both
    // k_direct2d_x2 and k_direct2d_x2s
    const int ty_k[2] = { 1, 2 };
    int *ord[2] = { nullptr, nullptr };              // tile orders for ty_k[0] and ty_k[1]
    int nt[2] = { 0, 0 }, bc[X2_VARIANTS] = { 0, 0, 0, 0 };
    float ms[X2_VARIANTS] = { 0.f, 0.f, 0.f, 0.f };
    float *u = nullptr, *lu = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool tune = p->N <= ((int64_t)1 << 24);
    nl_status s = NL_OK;
    // untuned (very large grids): x2s with TY = 2 (variant 1), x2 with TY = 1 (variant 0)
    int best = sym ? 1 : 0;
    for (int k = 0; k < 2 && s == NL_OK; ++k)
        if (tune || ty_k[k] == var_ty[best]) s = x2_order_for(p, ty_k[k], &ord[k], &nt[k], st);
    if (s == NL_OK && tune) {
        const DirectArgs a = make_args(p, NL_F32);
        if (cudaMalloc(&u, p->N * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&lu, p->N * sizeof(float)) != cudaSuccess ||
            cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
            cudaMemsetAsync(u, 0, p->N * sizeof(float), st) != cudaSuccess) {
            s = nl_cuda_fail(cudaErrorMemoryAllocation, "direct kernel tuning");
        }
        auto run = [&](int v) {
            const int k = var_ty[v] == ty_k[0] ? 0 : 1;
            return sym ? x2s_launch_any(p, v, a, u, lu, 1, ord[k], nt[k], &bc[v], st)
                       : (kap ? x2_launch_any<true>(p, v, a, u, lu, 1, ord[k], nt[k], &bc[v], st)
                              : x2_launch_any<false>(p, v, a, u, lu, 1, ord[k], nt[k], &bc[v], st));
        };
        if (s == NL_OK) s = time_variants(nvar, run, ms, e0, e1, st);
        best = 0;
        for (int v = 1; v < nvar; ++v) if (ms[v] < ms[best]) best = v;
    }
    if (u) cudaFree(u);
    if (lu) cudaFree(lu);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    const int kb = var_ty[best] == ty_k[0] ? 0 : 1;
    if (ord[1 - kb]) cudaFree(ord[1 - kb]);
    if (s != NL_OK) {
        if (ord[kb]) cudaFree(ord[kb]);
        return s;
    }
    p->x2_order = ord[kb];
    p->x2_tiles = nt[kb];
    p->x2_blocks = bc[best];
    p->x2_var = best;
    p->device_bytes += (size_t)nt[kb] * sizeof(int) + 2 * sizeof(int);
    if (sym) {
        // the pair kernel's 32 x (X2R_TY RB_P) tiles and its queue
        NL_CUDA_TRY(cudaMalloc(&p->x2r_queue, 2 * sizeof(int)));
        NL_CUDA_TRY(cudaMemsetAsync(p->x2r_queue, 0, 2 * sizeof(int), st));
        const nl_status so = x2_order_for(p, X2R_TY, &p->x2r_order, &p->x2r_tiles, st, 32);
        if (so != NL_OK) return so;
        p->device_bytes += (size_t)p->x2r_tiles * sizeof(int) + 2 * sizeof(int);
        const int rm = p->Rmax <= 4 ? 4 : p->Rmax <= 8 ? 8 : p->Rmax <= 16 ? 16 : p->Rmax <= 24 ? 24 : 32;
        NL_CUDA_TRY(cudaMalloc(&p->x2r_c32, p->N * sizeof(float)));
        NL_CUDA_TRY(cudaMalloc(&p->x2r_tp1, p->N * sizeof(float)));
        NL_CUDA_TRY(cudaMalloc(&p->x2r_jmin, (size_t)p->x2r_tiles * sizeof(int)));
        p->device_bytes += 2 * p->N * sizeof(float) + (size_t)p->x2r_tiles * sizeof(int);
        k_x2r_planes<<<(unsigned)((p->N + 255) / 256), 256, 0, st>>>(p->N, p->wh32, p->b32, p->thr,
                                                                    p->x2r_c32, p->x2r_tp1);
        k_x2r_tile_jmin<<<(unsigned)p->x2r_tiles, 256, 0, st>>>(p->n, (p->n + 31) / 32,
                                                                X2R_TY * RB_P, rm, p->thr,
                                                                p->x2r_jmin);
        NL_CUDA_TRY(cudaGetLastError());
        NL_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return NL_OK;
}
