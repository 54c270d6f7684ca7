// nl_net.cu -- the learned CG preconditioner (a project addition; the paper only remarks
// that the fast product can serve a Krylov method).
//
//   x = D^{-1} r / s,  s = RMS(D^{-1} r) per right-hand side
//   y1 = relu(conv1 x), y2 = relu(conv2 y1), o = conv3 y2     (3x3, zero padding, no bias,
//   M(r) = s (x + o)                                           channels 1 -> 32 -> 32 -> 1)
//
// Two-level form (nl_net_set_coarse with a block size b >= 2): the three layers without
// activations are one linear map K on a coarse grid of ceil(n/b)^2 cells, R sums each b x b
// block, P = R^T copies a cell to its block, and
//   M(r) = D^{-1} r + gamma P K^T K R r,   gamma = 1 / (b^2 mean(diag A)),
// symmetric positive definite for any weights.  K^T is the adjoint chain (the transposed
// weight layouts); training on the energy norm needs K applied to R r and to the coarse
// gradient, and one backward pass over both (d <g, K^T K x> = <K g, dK x> + <K x, dK g>).
//
// Weights are kept as FP32 masters (Adam) and used as bfloat16 (rounded to nearest even);
// activations and accumulation are FP32.  A 3x3 convolution tile of 16 x 16 pixels stages its
// (16+2)^2 x CIN input halo and its CIN x 9 x COUT weights in shared memory; each thread owns
// one pixel and COUT accumulators and reads weights as warp-uniform broadcasts.  The weight
// gradient is a per-tile partial contraction over the tile's pixels followed by a fixed-order
// reduction over tiles (deterministic).
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>

#include "nl_internal.cuh"

#define NL_NET_MAGIC 0x4e4c4e54u   // "NLNT"

namespace {

constexpr int TILE = 16;
constexpr int HALO = TILE + 2;
constexpr int NP1 = 32 * 1 * 9, NP2 = 32 * 32 * 9, NP3 = 1 * 32 * 9;
constexpr int NPARAM = NP1 + NP2 + NP3;
constexpr int OFF1 = 0, OFF2 = NP1, OFF3 = NP1 + NP2;
constexpr int RB = 256, NB = 152;

// ---------------------------------------------------------------------------
// 3x3 convolution: out[b][o][y][x] = sum_{c,dy,dx} wk[c][dy*3+dx][o] in[b][c][y+dy-1][x+dx-1]
// EPI 0: plain, 1: relu, 2: multiply by (mask > 0)
// ---------------------------------------------------------------------------
template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(256) k_conv3(const float *__restrict__ in,
                                               const float *__restrict__ wk,
                                               float *__restrict__ out,
                                               const float *__restrict__ mask, int H, int W)
{
    extern __shared__ __align__(16) float sm[];
    float *s_in = sm;                          // [CIN][HALO][HALO]
    float *s_w = sm + CIN * HALO * HALO;       // [CIN*9][COUT]
    const int b = blockIdx.z;
    const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE;
    const int tid = threadIdx.x;
    const size_t plane = (size_t)H * W;
    const float *inb = in + (size_t)b * CIN * plane;
    for (int e = tid; e < CIN * HALO * HALO; e += 256) {
        const int c = e / (HALO * HALO), rem = e % (HALO * HALO);
        const int gy = y0 - 1 + rem / HALO, gx = x0 - 1 + rem % HALO;
        s_in[e] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? inb[c * plane + (size_t)gy * W + gx] : 0.f;
    }
    for (int e = tid; e < CIN * 9 * COUT; e += 256) s_w[e] = wk[e];
    __syncthreads();
    const int tx = tid % TILE, ty = tid / TILE;
    float acc[COUT];
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[o] = 0.f;
    for (int c = 0; c < CIN; ++c) {
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const float v = s_in[c * HALO * HALO + (ty + t / 3) * HALO + tx + t % 3];
            const float *wr = s_w + (c * 9 + t) * COUT;
#pragma unroll
            for (int o = 0; o < COUT; ++o) acc[o] = fmaf(wr[o], v, acc[o]);
        }
    }
    const int gy = y0 + ty, gx = x0 + tx;
    if (gy >= H || gx >= W) return;
    float *ob = out + (size_t)b * COUT * plane + (size_t)gy * W + gx;
    const float *mb = (EPI == 2) ? mask + (size_t)b * COUT * plane + (size_t)gy * W + gx : nullptr;
#pragma unroll
    for (int o = 0; o < COUT; ++o) {
        float v = acc[o];
        if (EPI == 1) v = fmaxf(v, 0.f);
        if (EPI == 2) v = (mb[o * plane] > 0.f) ? v : 0.f;
        ob[o * plane] = v;
    }
}

// Weight gradient partials: part[blk][c][t][o] = sum over the tile's pixels of
// in[c][p + off(t)] * g[o][p].  Thread (c, og) owns 9 taps x OG outputs.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_conv3_wgrad(const float *__restrict__ in,
                                                     const float *__restrict__ g,
                                                     float *__restrict__ part, int H, int W)
{
    constexpr int OG = COUT < 4 ? COUT : 4;
    constexpr int NG = COUT / OG;
    extern __shared__ __align__(16) float sm[];
    float *s_in = sm;                          // [CIN][HALO][HALO]
    float *s_g = sm + CIN * HALO * HALO;       // [COUT][TILE*TILE]
    const int b = blockIdx.z;
    const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE;
    const int tid = threadIdx.x;
    const size_t plane = (size_t)H * W;
    const float *inb = in + (size_t)b * CIN * plane;
    const float *gb = g + (size_t)b * COUT * plane;
    for (int e = tid; e < CIN * HALO * HALO; e += 256) {
        const int c = e / (HALO * HALO), rem = e % (HALO * HALO);
        const int gy = y0 - 1 + rem / HALO, gx = x0 - 1 + rem % HALO;
        s_in[e] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? inb[c * plane + (size_t)gy * W + gx] : 0.f;
    }
    for (int e = tid; e < COUT * TILE * TILE; e += 256) {
        const int o = e / (TILE * TILE), p = e % (TILE * TILE);
        const int gy = y0 + p / TILE, gx = x0 + p % TILE;
        s_g[e] = (gy < H && gx < W) ? gb[o * plane + (size_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
    const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    float *pb = part + blk * (size_t)(CIN * 9 * COUT);
    for (int job = tid; job < CIN * NG; job += 256) {
        const int c = job / NG, og = job % NG;
        float acc[9][OG];
#pragma unroll
        for (int t = 0; t < 9; ++t)
#pragma unroll
            for (int k = 0; k < OG; ++k) acc[t][k] = 0.f;
        for (int p = 0; p < TILE * TILE; ++p) {
            const int py = p / TILE, px = p % TILE;
            float gv[OG];
#pragma unroll
            for (int k = 0; k < OG; ++k) gv[k] = s_g[(og * OG + k) * TILE * TILE + p];
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const float v = s_in[c * HALO * HALO + (py + t / 3) * HALO + px + t % 3];
#pragma unroll
                for (int k = 0; k < OG; ++k) acc[t][k] = fmaf(v, gv[k], acc[t][k]);
            }
        }
#pragma unroll
        for (int t = 0; t < 9; ++t)
#pragma unroll
            for (int k = 0; k < OG; ++k) pb[(c * 9 + t) * COUT + og * OG + k] = acc[t][k];
    }
}

// fixed-order reduction of the partials of one layer into the gradient ([o][c][3][3] layout)
__global__ void k_wgrad_reduce(const float *__restrict__ part, int nblk, int cin, int cout,
                               float *__restrict__ grad)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;    // kernel-layout index [c][t][o]
    const int P = cin * 9 * cout;
    if (k >= P) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * P + k];
    const int c = k / (9 * cout), t = (k / cout) % 9, o = k % cout;
    grad[(o * cin + c) * 9 + t] = s;
}

// bf16 weights -> per-layer forward [c][t][o] and backward-data [o][8-t][c] float layouts
__global__ void k_layouts(const __nv_bfloat16 *__restrict__ wb, float *__restrict__ wk,
                          float *__restrict__ wkt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NPARAM) return;
    int off, cin, cout, j;
    if (k < OFF2) { off = OFF1; cin = 1; cout = 32; }
    else if (k < OFF3) { off = OFF2; cin = 32; cout = 32; }
    else { off = OFF3; cin = 32; cout = 1; }
    j = k - off;                                    // [o][c][t]
    const int o = j / (cin * 9), c = (j / 9) % cin, t = j % 9;
    const float w = __bfloat162float(wb[k]);
    wk[off + (c * 9 + t) * cout + o] = w;
    wkt[off + (o * 9 + (8 - t)) * cin + c] = w;
}

// per sample: loss over the interior and d loss / d o
__global__ void __launch_bounds__(RB) k_loss(const float *__restrict__ x,
                                             const float *__restrict__ o,
                                             const float *__restrict__ e, float *__restrict__ go,
                                             float *__restrict__ loss, int S, int margin, int B)
{
    __shared__ double sh[2][RB / 32];
    const int b = blockIdx.x;
    const size_t base = (size_t)b * S * S;
    double ee = 0.0, dd = 0.0;
    for (int p = threadIdx.x; p < S * S; p += RB) {
        const int py = p / S, px = p % S;
        const bool in = py >= margin && py < S - margin && px >= margin && px < S - margin;
        if (!in) continue;
        const double ev = e[base + p], dv = (double)x[base + p] + o[base + p] - ev;
        ee += ev * ev;
        dd += dv * dv;
    }
    for (int k = 16; k > 0; k >>= 1) {
        ee += __shfl_down_sync(0xffffffffu, ee, k);
        dd += __shfl_down_sync(0xffffffffu, dd, k);
    }
    if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = ee; sh[1][threadIdx.x >> 5] = dd; }
    __syncthreads();
    double E = 0.0, Dd = 0.0;
    for (int w = 0; w < RB / 32; ++w) { E += sh[0][w]; Dd += sh[1][w]; }
    const double inv = E > 0.0 ? 1.0 / E : 0.0;
    if (threadIdx.x == 0) loss[b] = (float)(Dd * inv);
    for (int p = threadIdx.x; p < S * S; p += RB) {
        const int py = p / S, px = p % S;
        const bool in = py >= margin && py < S - margin && px >= margin && px < S - margin;
        const double dv = (double)x[base + p] + o[base + p] - e[base + p];
        go[base + p] = in ? (float)(2.0 * dv * inv / B) : 0.f;
    }
}

__global__ void k_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, __nv_bfloat16 *__restrict__ wb, float lr,
                       float c1, float c2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NPARAM) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float wk = w[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    w[k] = wk;
    wb[k] = __float2bfloat16_rn(wk);
}

__global__ void k_to_bf16(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NPARAM) wb[k] = __float2bfloat16_rn(w[k]);
}

// gather training crops: xb[b] = x[field][y0.., x0..], eb likewise
// (a crop outside the fields is written as zeros)
__global__ void k_gather_crops(const float *__restrict__ x, const float *__restrict__ e,
                               const int *__restrict__ crops, int nfields, int n, int S,
                               float *xb, float *eb)
{
    const int b = blockIdx.y;
    const int f = crops[3 * b], y0 = crops[3 * b + 1], x0 = crops[3 * b + 2];
    const bool ok = f >= 0 && f < nfields && y0 >= 0 && x0 >= 0 && y0 + S <= n && x0 + S <= n;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < S * S; p += gridDim.x * blockDim.x) {
        float xv = 0.f, ev = 0.f;
        if (ok) {
            const size_t src = (size_t)f * n * n + (size_t)(y0 + p / S) * n + x0 + p % S;
            xv = x[src];
            ev = e[src];
        }
        xb[(size_t)b * S * S + p] = xv;
        eb[(size_t)b * S * S + p] = ev;
    }
}

// ---- inference helpers ----
__global__ void __launch_bounds__(RB) k_prep_partial(const double *__restrict__ r,
                                                     const double *__restrict__ dinv, int64_t N,
                                                     double *__restrict__ part)
{
    const int rhs = blockIdx.y;
    double s = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)RB + threadIdx.x; k < N; k += (int64_t)NB * RB) {
        const double v = dinv[k] * r[(size_t)rhs * N + k];
        s += v * v;
    }
    __shared__ double sh[RB / 32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < RB / 32; ++w) t += sh[w];
        part[(size_t)rhs * NB + blockIdx.x] = t;
    }
}

__device__ __forceinline__ double fold_rms(const double *part, int rhs, int64_t N)
{
    double s = 0.0;
    for (int k = 0; k < NB; ++k) s += part[(size_t)rhs * NB + k];
    return sqrt(s / (double)N);
}

__global__ void k_prep_scale(const double *__restrict__ r, const double *__restrict__ dinv,
                             int64_t N, const double *__restrict__ part, float *__restrict__ xf)
{
    const int rhs = blockIdx.y;
    __shared__ double s_inv;
    if (threadIdx.x == 0) {
        const double s = fold_rms(part, rhs, N);
        s_inv = s > 0.0 ? 1.0 / s : 0.0;
    }
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x)
        xf[(size_t)rhs * N + k] = (float)(dinv[k] * r[(size_t)rhs * N + k] * s_inv);
}

__global__ void k_finish(const double *__restrict__ r, const double *__restrict__ dinv, int64_t N,
                         const double *__restrict__ part, const float *__restrict__ o,
                         double *__restrict__ z)
{
    const int rhs = blockIdx.y;
    __shared__ double s_s;
    if (threadIdx.x == 0) s_s = fold_rms(part, rhs, N);
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const size_t g = (size_t)rhs * N + k;
        z[g] = dinv[k] * r[g] + s_s * (double)o[g];
    }
}

// training pairs: x = D^{-1} r / s, e / s with s = RMS(D^{-1} r) of each field
__global__ void k_pairs(const double *__restrict__ r, const double *__restrict__ e,
                        const double *__restrict__ dinv, int64_t N,
                        const double *__restrict__ part, float *__restrict__ xo,
                        float *__restrict__ eo)
{
    const int f = blockIdx.y;
    __shared__ double s_inv;
    if (threadIdx.x == 0) {
        const double s = fold_rms(part, f, N);
        s_inv = s > 0.0 ? 1.0 / s : 0.0;
    }
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const size_t g = (size_t)f * N + k;
        xo[g] = (float)(dinv[k] * r[g] * s_inv);
        eo[g] = (float)(e[g] * s_inv);
    }
}

// energy-norm training: gather whole fields, r~ = x / dinv (the scaled residual)
__global__ void k_gather_fields(const float *__restrict__ x, const float *__restrict__ e,
                                const int *__restrict__ fields, int nfields, int64_t N,
                                const double *__restrict__ dinv, float *xb, float *eb, float *rb)
{
    const int b = blockIdx.y;
    const int f = fields[b];
    const bool ok = f >= 0 && f < nfields;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        float xv = 0.f, ev = 0.f;
        if (ok) { xv = x[(size_t)f * N + k]; ev = e[(size_t)f * N + k]; }
        xb[(size_t)b * N + k] = xv;
        eb[(size_t)b * N + k] = ev;
        rb[(size_t)b * N + k] = (float)((double)xv / dinv[k]);
    }
}

// z = x + o (the preconditioned step, scaled units)
__global__ void k_add(int64_t n, const float *__restrict__ a, const float *__restrict__ b, float *c)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) c[i] = a[i] + b[i];
}

// partial sums per field: z.Az (Az = -Lz), z.r, e.r
__global__ void __launch_bounds__(RB) k_energy_partial(const float *__restrict__ z,
                                                       const float *__restrict__ Lz,
                                                       const float *__restrict__ r,
                                                       const float *__restrict__ e, int64_t N,
                                                       double *__restrict__ part)
{
    __shared__ double sh[3][RB / 32];
    const int b = blockIdx.y;
    double zaz = 0.0, zr = 0.0, er = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)RB + threadIdx.x; k < N; k += (int64_t)NB * RB) {
        const size_t g = (size_t)b * N + k;
        zaz -= (double)z[g] * Lz[g];
        zr += (double)z[g] * r[g];
        er += (double)e[g] * r[g];
    }
    for (int o = 16; o > 0; o >>= 1) {
        zaz += __shfl_down_sync(0xffffffffu, zaz, o);
        zr += __shfl_down_sync(0xffffffffu, zr, o);
        er += __shfl_down_sync(0xffffffffu, er, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = zaz; sh[1][threadIdx.x >> 5] = zr; sh[2][threadIdx.x >> 5] = er;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, c = 0, d = 0;
        for (int w = 0; w < RB / 32; ++w) { a += sh[0][w]; c += sh[1][w]; d += sh[2][w]; }
        double *q = part + ((size_t)b * NB + blockIdx.x) * 3;
        q[0] = a; q[1] = c; q[2] = d;
    }
}

// loss_b = (z.Az - 2 z.r + e.r) / e.r ;  go = 2 (Az - r) / (e.r B)
__global__ void k_energy_grad(const float *__restrict__ Lz, const float *__restrict__ r, int64_t N,
                              const double *__restrict__ part, int B, float *__restrict__ go,
                              float *__restrict__ loss)
{
    const int b = blockIdx.y;
    __shared__ double s_inv;
    if (threadIdx.x == 0) {
        double a = 0, c = 0, d = 0;
        for (int k = 0; k < NB; ++k) {
            const double *q = part + ((size_t)b * NB + k) * 3;
            a += q[0]; c += q[1]; d += q[2];
        }
        s_inv = d > 0.0 ? 1.0 / d : 0.0;
        if (blockIdx.x == 0) loss[b] = (float)((a - 2.0 * c + d) * s_inv);
    }
    __syncthreads();
    const double scale = 2.0 * s_inv / B;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const size_t g = (size_t)b * N + k;
        go[g] = (float)(scale * (-(double)Lz[g] - (double)r[g]));
    }
}

// ---- two-level form ----
// rc[b][cell] = sum of v over the cell's b x b block (FP64 sum in a fixed order), times scale
template <typename T>
__global__ void __launch_bounds__(RB) k_restrict(const T *__restrict__ v, int n, int blk, int nc,
                                                 double scale, float *__restrict__ rc)
{
    __shared__ double sh[RB / 32];
    const int cell = blockIdx.x, b = blockIdx.y;
    const int cy = cell / nc, cx = cell % nc;
    const int y0 = cy * blk, x0 = cx * blk;
    const int hy = min(blk, n - y0), hx = min(blk, n - x0);
    const T *vb = v + (size_t)b * n * n;
    double s = 0.0;
    for (int k = threadIdx.x; k < hy * hx; k += RB)
        s += (double)vb[(size_t)(y0 + k / hx) * n + x0 + k % hx];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < RB / 32; ++w) t += sh[w];
        rc[(size_t)b * nc * nc + cell] = (float)(t * scale);
    }
}

// z = D^{-1} r + gamma P zc (FP64, inference)
__global__ void k_prolong_jacobi(const double *__restrict__ r, const double *__restrict__ dinv,
                                 const float *__restrict__ zc, int n, int blk, int nc,
                                 double gamma, double *__restrict__ z)
{
    const int b = blockIdx.y;
    const int64_t N = (int64_t)n * n;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(k / n), x = (int)(k % n);
        const size_t g = (size_t)b * N + k;
        z[g] = dinv[k] * r[g] + gamma * (double)zc[(size_t)b * nc * nc + (y / blk) * nc + x / blk];
    }
}

// z = x + gamma P zc (FP32, training; x = D^{-1} r in scaled units)
__global__ void k_prolong_add(const float *__restrict__ x, const float *__restrict__ zc, int n,
                              int blk, int nc, float gamma, float *__restrict__ z)
{
    const int b = blockIdx.y;
    const int64_t N = (int64_t)n * n;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(k / n), xx = (int)(k % n);
        const size_t g = (size_t)b * N + k;
        z[g] = x[g] + gamma * zc[(size_t)b * nc * nc + (y / blk) * nc + xx / blk];
    }
}

// Restriction by columns for n <= RC_MAXN: block (cy, b) sums each fine column over the
// cell row's blk rows (coalesced, thread per column), then each cell's blk column sums in
// order.  Same values as k_restrict up to the order of the FP64 sums.
constexpr int RC_MAXN = 4096;

template <typename T>
__global__ void __launch_bounds__(256) k_restrict_rows(const T *__restrict__ v, int n, int blk,
                                                       int nc, double scale,
                                                       float *__restrict__ rc)
{
    __shared__ double col[RC_MAXN];
    const int cy = blockIdx.x, b = blockIdx.y;
    const int y0 = cy * blk, y1 = min(n, y0 + blk);
    const T *vb = v + (size_t)b * n * n;
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        double s = 0.0;
#pragma unroll 8
        for (int y = y0; y < y1; ++y) s += (double)vb[(size_t)y * n + x];
        col[x] = s;
    }
    __syncthreads();
    for (int cx = threadIdx.x; cx < nc; cx += blockDim.x) {
        const int x0 = cx * blk, x1 = min(n, x0 + blk);
        double s = 0.0;
        for (int x = x0; x < x1; ++x) s += col[x];
        rc[(size_t)b * nc * nc + cy * nc + cx] = (float)(s * scale);
    }
}

// Coarse operator of the two-level form as a matrix: the network K is linear, so K^T K is a
// fixed m x m matrix on the coarse grid (m = nc^2 cells).  With H[i] = K e_i (the forward
// chain applied to the unit vectors) G[i][j] = H[i] . H[j]; both entries of a symmetric pair
// run the same products in the same order, so G is exactly symmetric.  FP64 sums.
constexpr int GRAM_MAXNC = 16;

__global__ void k_eye(float *__restrict__ e, int m)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m * m; k += gridDim.x * blockDim.x)
        e[k] = (k / m == k % m) ? 1.f : 0.f;
}

__global__ void k_gram(const float *__restrict__ h, int m, float *__restrict__ g)
{
    const int i = blockIdx.x;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < m; ++k) s = fma((double)h[(size_t)i * m + k], (double)h[(size_t)j * m + k], s);
        g[(size_t)i * m + j] = (float)s;
    }
}

// zc[b] = G rc[b]: one warp per row of G (held in registers), eight right-hand sides per block
__global__ void __launch_bounds__(256) k_coarse_gemv(const float *__restrict__ g,
                                                     const float *__restrict__ rc, int m, int nrhs,
                                                     float *__restrict__ zc)
{
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= m) return;
    float gr[GRAM_MAXNC * GRAM_MAXNC / 32];
#pragma unroll
    for (int q = 0; q < GRAM_MAXNC * GRAM_MAXNC / 32; ++q) {
        const int k = lane + 32 * q;
        gr[q] = k < m ? g[(size_t)i * m + k] : 0.f;
    }
    const int b1 = min(nrhs, (int)(blockIdx.y + 1) * 8);
    for (int b = blockIdx.y * 8; b < b1; ++b) {
        const float *x = rc + (size_t)b * m;
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < GRAM_MAXNC * GRAM_MAXNC / 32; ++q) {
            const int k = lane + 32 * q;
            if (k < m) s = fmaf(gr[q], x[k], s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) zc[(size_t)b * m + i] = s;
    }
}

}  // namespace

struct nl_net {
    uint32_t magic;
    int block;                           // 0: local form; >= 2: two-level with b x b blocks
    float *w32, *m, *v, *grad;
    __nv_bfloat16 *wb;
    float *wk, *wkt;
    int t;
    float *train;  size_t train_elems;   // training activations
    float *part;   size_t part_elems;    // weight-gradient partials
    float *loss;   int loss_elems;
    float *inf;    size_t inf_elems;     // inference activations
    double *red;   int red_elems;
    float *gram;   size_t gram_elems;    // G = K^T K on the coarse grid (two-level form)
    int gram_nc;                         // coarse size G was built for (0: none)
    uint64_t gram_ver;                   // weight version G was built from
    uint64_t wver;                       // weight version (bumped whenever wk/wkt change)
    uint64_t gen;                        // bumped whenever a buffer an apply uses moves
};

// Generations are unique across networks, so a network created at a freed one's address
// never matches a graph captured over the old one.
static uint64_t next_generation()
{
    static std::atomic<uint64_t> counter{0};
    return ++counter;
}

template <typename K>
static cudaError_t smem_attr(K kern, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static size_t conv_smem(int cin, int cout) { return sizeof(float) * (cin * HALO * HALO + cin * 9 * cout); }
static size_t wgrad_smem(int cin, int cout) { return sizeof(float) * (cin * HALO * HALO + cout * TILE * TILE); }

static nl_status net_attrs()
{
    static bool done = false;
    if (done) return NL_OK;
    NL_CUDA_TRY(smem_attr(k_conv3<32, 32, 1>, conv_smem(32, 32)));
    NL_CUDA_TRY(smem_attr(k_conv3<32, 32, 2>, conv_smem(32, 32)));
    NL_CUDA_TRY(smem_attr(k_conv3<32, 32, 0>, conv_smem(32, 32)));
    NL_CUDA_TRY(smem_attr(k_conv3<32, 1, 0>, conv_smem(32, 1)));
    NL_CUDA_TRY(smem_attr(k_conv3_wgrad<32, 32>, wgrad_smem(32, 32)));
    NL_CUDA_TRY(smem_attr(k_conv3_wgrad<32, 1>, wgrad_smem(32, 1)));
    done = true;
    return NL_OK;
}

static bool net_ok(const nl_net *n) { return n && n->magic == NL_NET_MAGIC; }

template <typename T>
static nl_status grow(T **buf, size_t *have, size_t need)
{
    if (*have >= need) return NL_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc((void **)buf, need * sizeof(T));
    if (e != cudaSuccess) {
        nl_set_error("network workspace allocation of %zu bytes failed", need * sizeof(T));
        return NL_ENOMEM;
    }
    *have = need;
    return NL_OK;
}

extern "C" nl_status nl_net_create(nl_net **out, const float *weights, void *stream)
{
    if (!out || !weights) {
        nl_set_error("nl_net_create: null argument");
        return NL_EINVAL;
    }
    *out = nullptr;
    for (int k = 0; k < NPARAM; ++k)
        if (!std::isfinite(weights[k])) {
            nl_set_error("nl_net_create: weight %d is not finite", k);
            return NL_EINVAL;
        }
    nl_status s = net_attrs();
    if (s != NL_OK) return s;
    nl_net *n = (nl_net *)calloc(1, sizeof(nl_net));
    if (!n) return NL_ENOMEM;
    n->magic = NL_NET_MAGIC;
    n->gen = next_generation();
    cudaError_t e = cudaSuccess;
    void **bufs[] = { (void **)&n->w32, (void **)&n->m, (void **)&n->v, (void **)&n->grad,
                      (void **)&n->wk, (void **)&n->wkt };
    for (void **b : bufs)
        if (e == cudaSuccess) e = cudaMalloc(b, NPARAM * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&n->wb, NPARAM * sizeof(__nv_bfloat16));
    if (e != cudaSuccess) {
        nl_net_destroy(n);
        nl_set_error("nl_net_create: allocation failed");
        return NL_ENOMEM;
    }
    cudaStream_t st = nl_stream(stream);
    NL_CUDA_TRY(cudaMemcpyAsync(n->w32, weights, NPARAM * sizeof(float), cudaMemcpyHostToDevice, st));
    NL_CUDA_TRY(cudaMemsetAsync(n->m, 0, NPARAM * sizeof(float), st));
    NL_CUDA_TRY(cudaMemsetAsync(n->v, 0, NPARAM * sizeof(float), st));
    k_to_bf16<<<(NPARAM + 255) / 256, 256, 0, st>>>(n->w32, n->wb);
    k_layouts<<<(NPARAM + 255) / 256, 256, 0, st>>>(n->wb, n->wk, n->wkt);
    ++n->wver;
    NL_CUDA_TRY(cudaGetLastError());
    NL_CUDA_TRY(cudaStreamSynchronize(st));
    *out = n;
    return NL_OK;
}

extern "C" nl_status nl_net_destroy(nl_net *n)
{
    if (!n) return NL_OK;
    if (!net_ok(n)) {
        nl_set_error("nl_net_destroy: not a network");
        return NL_EINVAL;
    }
    cudaDeviceSynchronize();
    void *ptrs[] = { n->w32, n->m, n->v, n->grad, n->wb, n->wk, n->wkt, n->train, n->part,
                     n->loss, n->inf, n->red, n->gram };
    for (void *q : ptrs) if (q) cudaFree(q);
    n->magic = 0;
    free(n);
    return NL_OK;
}

extern "C" nl_status nl_net_get_weights(nl_net *n, float *weights, void *stream)
{
    if (!net_ok(n) || !weights) {
        nl_set_error("nl_net_get_weights: bad argument");
        return NL_EINVAL;
    }
    cudaStream_t st = nl_stream(stream);
    NL_CUDA_TRY(cudaMemcpyAsync(weights, n->w32, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st));
    NL_CUDA_TRY(cudaStreamSynchronize(st));
    return NL_OK;
}

// forward through the three layers on [B][1][H][W] -> o [B][1][H][W]
static nl_status net_forward(nl_net *n, const float *x, float *y1, float *y2, float *o, int B,
                             int H, int W, cudaStream_t st)
{
    const dim3 grid((W + TILE - 1) / TILE, (H + TILE - 1) / TILE, B);
    k_conv3<1, 32, 1><<<grid, 256, conv_smem(1, 32), st>>>(x, n->wk + OFF1, y1, nullptr, H, W);
    k_conv3<32, 32, 1><<<grid, 256, conv_smem(32, 32), st>>>(y1, n->wk + OFF2, y2, nullptr, H, W);
    k_conv3<32, 1, 0><<<grid, 256, conv_smem(32, 1), st>>>(y2, n->wk + OFF3, o, nullptr, H, W);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

extern "C" nl_status nl_net_forward(nl_net *n, const float *x, float *o, int batch, int H, int W,
                                    void *stream)
{
    if (!net_ok(n) || !x || !o || batch < 1 || batch > 65535 || H < 1 || W < 1) {
        nl_set_error("nl_net_forward: bad argument");
        return NL_EINVAL;
    }
    const size_t plane = (size_t)H * W;
    nl_status s = grow(&n->inf, &n->inf_elems, 64 * plane * batch);
    if (s != NL_OK) return s;
    return net_forward(n, x, n->inf, n->inf + 32 * plane * batch, o, batch, H, W, nl_stream(stream));
}

extern "C" nl_status nl_net_train_step(nl_net *n, const float *x, const float *e, int nfields,
                                       int fn, const int *crops, int batch, int S, int margin,
                                       float lr, float *loss_host, void *stream)
{
    if (!net_ok(n) || !x || !e || !crops || batch < 1 || batch > 65535 || S < 4 ||
        margin < 0 || 2 * margin >= S || S > fn || nfields < 1 || !(lr > 0.f)) {
        nl_set_error("nl_net_train_step: bad argument");
        return NL_EINVAL;
    }
    cudaStream_t st = nl_stream(stream);
    const size_t plane = (size_t)S * S;
    // xb | eb | o | go | y1 | y2 | g2 | g1   (y1, y2, g2, g1: 32 channels)
    const size_t need = plane * batch * (4 + 4 * 32);
    nl_status s = grow(&n->train, &n->train_elems, need);
    if (s != NL_OK) return s;
    const int tiles = ((S + TILE - 1) / TILE) * ((S + TILE - 1) / TILE);
    const size_t nblk = (size_t)tiles * batch;
    s = grow(&n->part, &n->part_elems, nblk * NP2);
    if (s != NL_OK) return s;
    size_t le = (size_t)n->loss_elems;
    s = grow(&n->loss, &le, (size_t)batch);
    if (s != NL_OK) return s;
    n->loss_elems = (int)le;
    float *xb = n->train, *eb = xb + plane * batch, *o = eb + plane * batch, *go = o + plane * batch;
    float *y1 = go + plane * batch, *y2 = y1 + 32 * plane * batch;
    float *g2 = y2 + 32 * plane * batch, *g1 = g2 + 32 * plane * batch;

    k_gather_crops<<<dim3((unsigned)((plane + 255) / 256), batch), 256, 0, st>>>(x, e, crops, nfields, fn, S, xb, eb);
    if ((s = net_forward(n, xb, y1, y2, o, batch, S, S, st)) != NL_OK) return s;
    k_loss<<<batch, RB, 0, st>>>(xb, o, eb, go, n->loss, S, margin, batch);
    const dim3 grid((S + TILE - 1) / TILE, (S + TILE - 1) / TILE, batch);
    // layer 3: dW3 and g2 = conv3^T(go) masked by y2 > 0
    k_conv3_wgrad<32, 1><<<grid, 256, wgrad_smem(32, 1), st>>>(y2, go, n->part, S, S);
    k_wgrad_reduce<<<(NP3 + 255) / 256, 256, 0, st>>>(n->part, (int)nblk, 32, 1, n->grad + OFF3);
    k_conv3<1, 32, 2><<<grid, 256, conv_smem(1, 32), st>>>(go, n->wkt + OFF3, g2, y2, S, S);
    // layer 2: dW2 and g1 = conv2^T(g2) masked by y1 > 0
    k_conv3_wgrad<32, 32><<<grid, 256, wgrad_smem(32, 32), st>>>(y1, g2, n->part, S, S);
    k_wgrad_reduce<<<(NP2 + 255) / 256, 256, 0, st>>>(n->part, (int)nblk, 32, 32, n->grad + OFF2);
    k_conv3<32, 32, 2><<<grid, 256, conv_smem(32, 32), st>>>(g2, n->wkt + OFF2, g1, y1, S, S);
    // layer 1: dW1
    k_conv3_wgrad<1, 32><<<grid, 256, wgrad_smem(1, 32), st>>>(xb, g1, n->part, S, S);
    k_wgrad_reduce<<<(NP1 + 255) / 256, 256, 0, st>>>(n->part, (int)nblk, 1, 32, n->grad + OFF1);
    // Adam
    n->t += 1;
    const float c1 = 1.f - powf(0.9f, (float)n->t), c2 = 1.f - powf(0.999f, (float)n->t);
    k_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(n->w32, n->m, n->v, n->grad, n->wb, lr, c1, c2);
    k_layouts<<<(NPARAM + 255) / 256, 256, 0, st>>>(n->wb, n->wk, n->wkt);
    ++n->wver;
    NL_CUDA_TRY(cudaGetLastError());
    if (loss_host) {
        float tmp[1024];
        const int cnt = batch < 1024 ? batch : 1024;
        NL_CUDA_TRY(cudaMemcpyAsync(tmp, n->loss, cnt * sizeof(float), cudaMemcpyDeviceToHost, st));
        NL_CUDA_TRY(cudaStreamSynchronize(st));
        double sum = 0.0;
        for (int b = 0; b < cnt; ++b) sum += tmp[b];
        *loss_host = (float)(sum / cnt);
    }
    return NL_OK;
}

// plan-owned inverse Jacobi diagonal (FP64), computed once
static nl_status plan_dinv(nl_plan *p, cudaStream_t st, const double **out)
{
    if (!p->dinv64) {
        const int64_t per = p->family == NL_PD_BOND ? 2 * p->N : p->N;
        double *d = nullptr, *z = nullptr;
        if (cudaMalloc(&d, per * sizeof(double)) != cudaSuccess) return NL_ENOMEM;
        if (cudaMalloc(&z, per * sizeof(double)) != cudaSuccess) { cudaFree(d); return NL_ENOMEM; }
        NL_CUDA_TRY(cudaMemsetAsync(z, 0, per * sizeof(double), st));
        nl_status s = nl_diag_launch(p, z, d, st);
        if (s != NL_OK) { cudaFree(d); cudaFree(z); return s; }
        // mean of the diagonal on the host (fixed order), then invert in place
        double *h = (double *)malloc(per * sizeof(double));
        if (!h) { cudaFree(d); cudaFree(z); return NL_ENOMEM; }
        cudaError_t ce = cudaMemcpyAsync(h, d, per * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) { free(h); cudaFree(d); cudaFree(z); return nl_cuda_fail(ce, "diagonal"); }
        double sum = 0.0;
        for (int64_t k = 0; k < per; ++k) sum += h[k];
        free(h);
        p->diag_mean = sum / (double)per;
        nl_invert_launch(per, d, st);
        NL_CUDA_TRY(cudaStreamSynchronize(st));
        cudaFree(z);
        p->dinv64 = d;
        p->device_bytes += per * sizeof(double);
    }
    *out = p->dinv64;
    return NL_OK;
}

// shared backward pass + Adam for a batch of B planes of H x W
static nl_status net_backward_adam(nl_net *n, const float *xb, const float *y1, const float *y2,
                                   const float *go, float *g2, float *g1, int B, int H, int W,
                                   float lr, cudaStream_t st, bool relu = true)
{
    const int tiles = ((H + TILE - 1) / TILE) * ((W + TILE - 1) / TILE);
    const size_t nblk = (size_t)tiles * B;
    nl_status s = grow(&n->part, &n->part_elems, nblk * NP2);
    if (s != NL_OK) return s;
    const dim3 grid((W + TILE - 1) / TILE, (H + TILE - 1) / TILE, B);
    k_conv3_wgrad<32, 1><<<grid, 256, wgrad_smem(32, 1), st>>>(y2, go, n->part, H, W);
    k_wgrad_reduce<<<(NP3 + 255) / 256, 256, 0, st>>>(n->part, (int)nblk, 32, 1, n->grad + OFF3);
    if (relu) k_conv3<1, 32, 2><<<grid, 256, conv_smem(1, 32), st>>>(go, n->wkt + OFF3, g2, y2, H, W);
    else k_conv3<1, 32, 0><<<grid, 256, conv_smem(1, 32), st>>>(go, n->wkt + OFF3, g2, nullptr, H, W);
    k_conv3_wgrad<32, 32><<<grid, 256, wgrad_smem(32, 32), st>>>(y1, g2, n->part, H, W);
    k_wgrad_reduce<<<(NP2 + 255) / 256, 256, 0, st>>>(n->part, (int)nblk, 32, 32, n->grad + OFF2);
    if (relu) k_conv3<32, 32, 2><<<grid, 256, conv_smem(32, 32), st>>>(g2, n->wkt + OFF2, g1, y1, H, W);
    else k_conv3<32, 32, 0><<<grid, 256, conv_smem(32, 32), st>>>(g2, n->wkt + OFF2, g1, nullptr, H, W);
    k_conv3_wgrad<1, 32><<<grid, 256, wgrad_smem(1, 32), st>>>(xb, g1, n->part, H, W);
    k_wgrad_reduce<<<(NP1 + 255) / 256, 256, 0, st>>>(n->part, (int)nblk, 1, 32, n->grad + OFF1);
    n->t += 1;
    const float c1 = 1.f - powf(0.9f, (float)n->t), c2 = 1.f - powf(0.999f, (float)n->t);
    k_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(n->w32, n->m, n->v, n->grad, n->wb, lr, c1, c2);
    k_layouts<<<(NPARAM + 255) / 256, 256, 0, st>>>(n->wb, n->wk, n->wkt);
    ++n->wver;
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

// ---- two-level form: coarse geometry, K and K^T on [B][nc][nc] ----
static int coarse_n(const nl_net *n, const nl_plan *p) { return (p->n + n->block - 1) / n->block; }

static double two_level_gamma(const nl_net *n, const nl_plan *p)
{
    return 1.0 / ((double)n->block * n->block * p->diag_mean);
}

template <typename T>
static void launch_restrict(const T *v, int nn, int blk, int nc, double scale, float *rc, int B,
                            cudaStream_t st)
{
    if (nn <= RC_MAXN)
        k_restrict_rows<T><<<dim3((unsigned)nc, B), 256, 0, st>>>(v, nn, blk, nc, scale, rc);
    else
        k_restrict<T><<<dim3((unsigned)(nc * nc), B), RB, 0, st>>>(v, nn, blk, nc, scale, rc);
}

// grow() for buffers an apply reads: a move invalidates graphs captured over the old address
template <typename T>
static nl_status grow_tracked(nl_net *n, T **buf, size_t *have, size_t need)
{
    T *const old = *buf;
    const nl_status s = grow(buf, have, need);
    if (*buf != old) n->gen = next_generation();
    return s;
}

// u = K x, keeping the activations a1, a2 ([B][32][nc][nc])
static void chain_forward(nl_net *n, const float *x, float *a1, float *a2, float *u, int B, int nc,
                          cudaStream_t st)
{
    const dim3 grid((nc + TILE - 1) / TILE, (nc + TILE - 1) / TILE, B);
    k_conv3<1, 32, 0><<<grid, 256, conv_smem(1, 32), st>>>(x, n->wk + OFF1, a1, nullptr, nc, nc);
    k_conv3<32, 32, 0><<<grid, 256, conv_smem(32, 32), st>>>(a1, n->wk + OFF2, a2, nullptr, nc, nc);
    k_conv3<32, 1, 0><<<grid, 256, conv_smem(32, 1), st>>>(a2, n->wk + OFF3, u, nullptr, nc, nc);
}

// zc = K^T u (t2, t1: [B][32][nc][nc] scratch)
static void chain_adjoint(nl_net *n, const float *u, float *t2, float *t1, float *zc, int B, int nc,
                          cudaStream_t st)
{
    const dim3 grid((nc + TILE - 1) / TILE, (nc + TILE - 1) / TILE, B);
    k_conv3<1, 32, 0><<<grid, 256, conv_smem(1, 32), st>>>(u, n->wkt + OFF3, t2, nullptr, nc, nc);
    k_conv3<32, 32, 0><<<grid, 256, conv_smem(32, 32), st>>>(t2, n->wkt + OFF2, t1, nullptr, nc, nc);
    k_conv3<32, 1, 0><<<grid, 256, conv_smem(32, 1), st>>>(t1, n->wkt + OFF1, zc, nullptr, nc, nc);
}

// one energy-norm Adam step of the two-level form (see the header of this file)
static nl_status train_energy_two_level(nl_net *n, nl_plan *p, const float *x, const float *e,
                                        int nfields, const int *fields, int batch, float lr,
                                        const double *dinv, cudaStream_t st)
{
    const int64_t N = p->N;
    const int nn = p->n, blk = n->block, nc = coarse_n(n, p);
    const size_t f = (size_t)N * batch, c = (size_t)nc * nc, cb = c * batch;
    // fine: xb eb rb z Lz go | coarse: in[2B] a1[2B][32] a2[2B][32] uv[2B] up[2B] t2 t1 zc
    //        g2[2B][32] g1[2B][32]
    const size_t need = f * 6 + cb * (2 + 64 + 64 + 2 + 2 + 32 + 32 + 1 + 64 + 64);
    nl_status s = grow(&n->train, &n->train_elems, need);
    if (s != NL_OK) return s;
    float *xb = n->train, *eb = xb + f, *rb = eb + f, *z = rb + f, *Lz = z + f, *go = Lz + f;
    float *cin = go + f, *a1 = cin + 2 * cb, *a2 = a1 + 64 * cb, *uv = a2 + 64 * cb;
    float *up = uv + 2 * cb, *t2 = up + 2 * cb, *t1 = t2 + 32 * cb, *zc = t1 + 32 * cb;
    float *g2 = zc + cb, *g1 = g2 + 64 * cb;
    const double gam = two_level_gamma(n, p);
    const unsigned gx = (unsigned)((N + 255) / 256 < 1024 ? (N + 255) / 256 : 1024);
    k_gather_fields<<<dim3(gx, batch), 256, 0, st>>>(x, e, fields, nfields, N, dinv, xb, eb, rb);
    launch_restrict<float>(rb, nn, blk, nc, 1.0, cin, batch, st);
    chain_forward(n, cin, a1, a2, uv, batch, nc, st);                       // u = K R r
    chain_adjoint(n, uv, t2, t1, zc, batch, nc, st);                        // K^T u
    k_prolong_add<<<dim3(gx, batch), 256, 0, st>>>(xb, zc, nn, blk, nc, (float)gam, z);
    if ((s = nl_direct_launch(p, z, Lz, batch, NL_F32, st)) != NL_OK) return s;
    k_energy_partial<<<dim3(NB, batch), RB, 0, st>>>(z, Lz, rb, eb, N, n->red);
    k_energy_grad<<<dim3(gx, batch), 256, 0, st>>>(Lz, rb, N, n->red, batch, go, n->loss);
    launch_restrict<float>(go, nn, blk, nc, gam, cin + cb, batch, st);
    chain_forward(n, cin + cb, a1 + 32 * cb, a2 + 32 * cb, uv + cb, batch, nc, st);   // v = K g
    // upstream: the first half (inputs R r) takes v, the second (inputs g) takes u
    NL_CUDA_TRY(cudaMemcpyAsync(up, uv + cb, cb * sizeof(float), cudaMemcpyDeviceToDevice, st));
    NL_CUDA_TRY(cudaMemcpyAsync(up + cb, uv, cb * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return net_backward_adam(n, cin, a1, a2, up, g2, g1, 2 * batch, nc, nc, lr, st, false);
}

static nl_status train_energy_local(nl_net *n, nl_plan *p, const float *x, const float *e,
                                    int nfields, const int *fields, int batch, float lr,
                                    const double *dinv, cudaStream_t st);

extern "C" nl_status nl_net_train_step_energy(nl_net *n, nl_plan *p, const float *x,
                                              const float *e, int nfields, const int *fields,
                                              int batch, float lr, float *loss_host,
                                              void *stream)
{
    if (!net_ok(n) || !nl_plan_ok(p) || !x || !e || !fields || batch < 1 || batch > 1024 ||
        nfields < 1 || !(lr > 0.f)) {
        nl_set_error("nl_net_train_step_energy: bad argument");
        return NL_EINVAL;
    }
    if (p->d != 2 || p->family == NL_PD_BOND || !p->symmetric) {
        nl_set_error("nl_net_train_step_energy: needs the symmetric 2-D scalar operator");
        return NL_EUNSUPPORTED;
    }
    cudaStream_t st = nl_stream(stream);
    const double *dinv = nullptr;
    nl_status s = plan_dinv(p, st, &dinv);
    if (s != NL_OK) return s;
    const size_t f = (size_t)p->N * batch;
    size_t le = (size_t)n->loss_elems;
    if ((s = grow(&n->loss, &le, (size_t)batch)) != NL_OK) return s;
    n->loss_elems = (int)le;
    size_t re = (size_t)n->red_elems;
    if ((s = grow(&n->red, &re, (size_t)NB * batch * 3)) != NL_OK) return s;
    n->red_elems = (int)re;
    if (n->block >= 2) {
        s = train_energy_two_level(n, p, x, e, nfields, fields, batch, lr, dinv, st);
    } else {
        // xb eb rb o z Lz go | y1 y2 g2 g1 (32 channels each)
        if ((s = grow(&n->train, &n->train_elems, f * (7 + 4 * 32))) != NL_OK) return s;
        s = train_energy_local(n, p, x, e, nfields, fields, batch, lr, dinv, st);
    }
    if (s != NL_OK) return s;
    if (loss_host) {
        float tmp[1024];
        NL_CUDA_TRY(cudaMemcpyAsync(tmp, n->loss, batch * sizeof(float), cudaMemcpyDeviceToHost, st));
        NL_CUDA_TRY(cudaStreamSynchronize(st));
        double sum = 0.0;
        for (int b = 0; b < batch; ++b) sum += tmp[b];
        *loss_host = (float)(sum / batch);
    }
    return NL_OK;
}

// one energy-norm Adam step of the local form on whole fields
static nl_status train_energy_local(nl_net *n, nl_plan *p, const float *x, const float *e,
                                    int nfields, const int *fields, int batch, float lr,
                                    const double *dinv, cudaStream_t st)
{
    const int64_t N = p->N;
    const int H = p->n, W = p->n;
    const size_t f = (size_t)N * batch;
    nl_status s;
    float *xb = n->train, *eb = xb + f, *rb = eb + f, *o = rb + f, *z = o + f, *Lz = z + f;
    float *go = Lz + f, *y1 = go + f, *y2 = y1 + 32 * f, *g2 = y2 + 32 * f, *g1 = g2 + 32 * f;
    const unsigned gx = (unsigned)((N + 255) / 256 < 1024 ? (N + 255) / 256 : 1024);
    k_gather_fields<<<dim3(gx, batch), 256, 0, st>>>(x, e, fields, nfields, N, dinv, xb, eb, rb);
    if ((s = net_forward(n, xb, y1, y2, o, batch, H, W, st)) != NL_OK) return s;
    k_add<<<(unsigned)((f + 255) / 256), 256, 0, st>>>((int64_t)f, xb, o, z);
    if ((s = nl_direct_launch(p, z, Lz, batch, NL_F32, st)) != NL_OK) return s;
    k_energy_partial<<<dim3(NB, batch), RB, 0, st>>>(z, Lz, rb, eb, N, n->red);
    k_energy_grad<<<dim3(gx, batch), 256, 0, st>>>(Lz, rb, N, n->red, batch, go, n->loss);
    return net_backward_adam(n, xb, y1, y2, go, g2, g1, batch, H, W, lr, st);
}

extern "C" nl_status nl_net_gradient(nl_net *n, float *grad_host, void *stream)
{
    if (!net_ok(n) || !grad_host) {
        nl_set_error("nl_net_gradient: bad argument");
        return NL_EINVAL;
    }
    cudaStream_t st = nl_stream(stream);
    NL_CUDA_TRY(cudaMemcpyAsync(grad_host, n->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st));
    NL_CUDA_TRY(cudaStreamSynchronize(st));
    return NL_OK;
}

static size_t two_level_inf_elems(const nl_net *n, const nl_plan *p, int nrhs)
{
    const int nc = coarse_n(n, p);
    const size_t c = (size_t)nc * nc;
    if (nc <= GRAM_MAXNC) return c * nrhs * 2;              // rc zc
    return c * nrhs * (1 + 32 + 32 + 1 + 32 + 32 + 1);     // rc a1 a2 u t2 t1 zc
}

// Build G = K^T K for the current weights and coarse size (nothing to do when up to date).
// Allocates and synchronises: runs before a CG chunk is captured, never inside one.
static nl_status ensure_gram(nl_net *n, int nc, cudaStream_t st)
{
    if (n->gram_nc == nc && n->gram_ver == n->wver) return NL_OK;
    const size_t m = (size_t)nc * nc;
    nl_status s = grow_tracked(n, &n->gram, &n->gram_elems, m * m);
    if (s != NL_OK) return s;
    s = grow(&n->train, &n->train_elems, m * m * (1 + 32 + 32 + 1));
    if (s != NL_OK) return s;
    float *e = n->train, *a1 = e + m * m, *a2 = a1 + 32 * m * m, *h = a2 + 32 * m * m;
    k_eye<<<(unsigned)((m * m + 255) / 256), 256, 0, st>>>(e, (int)m);
    chain_forward(n, e, a1, a2, h, (int)m, nc, st);                         // H[i] = K e_i
    k_gram<<<(unsigned)m, 256, 0, st>>>(h, (int)m, n->gram);
    NL_CUDA_TRY(cudaGetLastError());
    n->gram_nc = nc;
    n->gram_ver = n->wver;
    return NL_OK;
}

nl_status nl_net_apply_launch(nl_net *n, nl_plan *p, const double *r, double *z, int nrhs,
                              cudaStream_t st)
{
    const double *dinv = nullptr;
    nl_status s = plan_dinv(p, st, &dinv);
    if (s != NL_OK) return s;
    if (n->block >= 2) {
        const int nc = coarse_n(n, p);
        const size_t cb = (size_t)nc * nc * nrhs;
        s = grow_tracked(n, &n->inf, &n->inf_elems, two_level_inf_elems(n, p, nrhs));
        if (s != NL_OK) return s;
        float *rc = n->inf, *zc;
        launch_restrict<double>(r, p->n, n->block, nc, 1.0, rc, nrhs, st);
        if (nc <= GRAM_MAXNC) {
            if ((s = ensure_gram(n, nc, st)) != NL_OK) return s;
            zc = rc + cb;
            const int m = nc * nc;
            k_coarse_gemv<<<dim3((unsigned)((m + 7) / 8), (unsigned)((nrhs + 7) / 8)), 256, 0, st>>>(
                n->gram, rc, m, nrhs, zc);
        } else {
            float *a1 = rc + cb, *a2 = a1 + 32 * cb, *u = a2 + 32 * cb;
            float *t2 = u + cb, *t1 = t2 + 32 * cb;
            zc = t1 + 32 * cb;
            chain_forward(n, rc, a1, a2, u, nrhs, nc, st);
            chain_adjoint(n, u, t2, t1, zc, nrhs, nc, st);
        }
        const unsigned gx = (unsigned)((p->N + 255) / 256 < 1024 ? (p->N + 255) / 256 : 1024);
        k_prolong_jacobi<<<dim3(gx, nrhs), 256, 0, st>>>(r, dinv, zc, p->n, n->block, nc,
                                                         two_level_gamma(n, p), z);
        NL_CUDA_TRY(cudaGetLastError());
        return NL_OK;
    }
    const int64_t N = p->N;
    const int H = p->n, W = p->n;
    s = grow_tracked(n, &n->inf, &n->inf_elems, (size_t)(66) * N * nrhs);
    if (s != NL_OK) return s;
    size_t re = (size_t)n->red_elems;
    s = grow_tracked(n, &n->red, &re, (size_t)NB * nrhs);
    if (s != NL_OK) return s;
    n->red_elems = (int)re;
    float *xf = n->inf, *o = xf + (size_t)N * nrhs, *y1 = o + (size_t)N * nrhs;
    float *y2 = y1 + (size_t)32 * N * nrhs;
    k_prep_partial<<<dim3(NB, nrhs), RB, 0, st>>>(r, dinv, N, n->red);
    const unsigned gx = (unsigned)((N + 255) / 256 < 1024 ? (N + 255) / 256 : 1024);
    k_prep_scale<<<dim3(gx, nrhs), 256, 0, st>>>(r, dinv, N, n->red, xf);
    if ((s = net_forward(n, xf, y1, y2, o, nrhs, H, W, st)) != NL_OK) return s;
    k_finish<<<dim3(gx, nrhs), 256, 0, st>>>(r, dinv, N, n->red, o, z);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

// Make sure the workspaces an apply needs exist (so a captured CG chunk allocates nothing).
nl_status nl_net_reserve(nl_net *n, nl_plan *p, int nrhs, cudaStream_t st)
{
    const double *dinv = nullptr;
    nl_status s = plan_dinv(p, st, &dinv);
    if (s != NL_OK) return s;
    s = grow_tracked(n, &n->inf, &n->inf_elems, n->block >= 2 ? two_level_inf_elems(n, p, nrhs)
                                                               : (size_t)66 * p->N * nrhs);
    if (s != NL_OK) return s;
    size_t re = (size_t)n->red_elems;
    s = grow_tracked(n, &n->red, &re, (size_t)NB * nrhs);
    n->red_elems = (int)re;
    if (s == NL_OK && n->block >= 2 && coarse_n(n, p) <= GRAM_MAXNC)
        s = ensure_gram(n, coarse_n(n, p), st);
    return s;
}

uint64_t nl_net_generation(const nl_net *n) { return n->gen; }

bool nl_net_valid(const nl_net *n) { return net_ok(n); }

extern "C" nl_status nl_net_apply(nl_net *n, nl_plan *p, const double *r, double *z, int nrhs,
                                  void *stream)
{
    if (!net_ok(n) || !nl_plan_ok(p) || !r || !z || nrhs < 1 || nrhs > 65535) {
        nl_set_error("nl_net_apply: bad argument");
        return NL_EINVAL;
    }
    if (p->d != 2 || p->family == NL_PD_BOND || !p->symmetric) {
        nl_set_error("nl_net_apply: the network preconditions the symmetric 2-D scalar operator");
        return NL_EUNSUPPORTED;
    }
    return nl_net_apply_launch(n, p, r, z, nrhs, nl_stream(stream));
}

extern "C" nl_status nl_net_prepare_pairs(nl_plan *p, const double *r, const double *e, int count,
                                          float *x_out, float *e_out, void *stream)
{
    if (!nl_plan_ok(p) || !r || !e || !x_out || !e_out || count < 1 || count > 65535) {
        nl_set_error("nl_net_prepare_pairs: bad argument");
        return NL_EINVAL;
    }
    if (p->d != 2 || p->family == NL_PD_BOND || !p->symmetric) {
        nl_set_error("nl_net_prepare_pairs: needs the symmetric 2-D scalar operator");
        return NL_EUNSUPPORTED;
    }
    cudaStream_t st = nl_stream(stream);
    const double *dinv = nullptr;
    nl_status s = plan_dinv(p, st, &dinv);
    if (s != NL_OK) return s;
    double *part = nullptr;
    if (cudaMalloc(&part, (size_t)NB * count * sizeof(double)) != cudaSuccess) return NL_ENOMEM;
    const int64_t N = p->N;
    k_prep_partial<<<dim3(NB, count), RB, 0, st>>>(r, dinv, N, part);
    const unsigned gx = (unsigned)((N + 255) / 256 < 1024 ? (N + 255) / 256 : 1024);
    k_pairs<<<dim3(gx, count), 256, 0, st>>>(r, e, dinv, N, part, x_out, e_out);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    cudaFree(part);
    if (ce != cudaSuccess) return nl_cuda_fail(ce, "nl_net_prepare_pairs");
    return NL_OK;
}

// r_k = f + (L H_k) (L H_k in r on entry), e_k = x - H_k, for k < count
__global__ void k_hist_residual(const double *__restrict__ f, const double *__restrict__ x,
                                const double *__restrict__ H, double *__restrict__ r,
                                double *__restrict__ e, int64_t N, int count)
{
    const int64_t tot = N * count;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < tot;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = g % N;
        r[g] += f[i];
        e[g] = x[i] - H[g];
    }
}

extern "C" nl_status nl_net_history_pairs(nl_plan *p, const double *f, const double *x,
                                          const double *history, int count, float *x_out,
                                          float *e_out, void *stream)
{
    if (!nl_plan_ok(p) || !f || !x || !history || !x_out || !e_out || count < 1 ||
        count > 65535) {
        nl_set_error("nl_net_history_pairs: bad argument");
        return NL_EINVAL;
    }
    if (p->d != 2 || p->family == NL_PD_BOND || !p->symmetric) {
        nl_set_error("nl_net_history_pairs: needs the symmetric 2-D scalar operator");
        return NL_EUNSUPPORTED;
    }
    cudaStream_t st = nl_stream(stream);
    const int64_t N = p->N;
    double *r = nullptr, *e = nullptr;
    if (cudaMalloc(&r, (size_t)count * N * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&e, (size_t)count * N * sizeof(double)) != cudaSuccess) {
        if (r) cudaFree(r);
        nl_set_error("nl_net_history_pairs: allocation of %d residual fields failed", count);
        return NL_ENOMEM;
    }
    nl_status s = nl_apply(p, history, r, count, NL_F64, stream);
    if (s == NL_OK) {
        const int64_t tot = (int64_t)count * N;
        const unsigned g = (unsigned)std::min<int64_t>((tot + 255) / 256, 4096);
        k_hist_residual<<<g, 256, 0, st>>>(f, x, history, r, e, N, count);
        const cudaError_t ce = cudaGetLastError();
        s = ce == cudaSuccess ? nl_net_prepare_pairs(p, r, e, count, x_out, e_out, stream)
                              : nl_cuda_fail(ce, "nl_net_history_pairs");
    }
    cudaStreamSynchronize(st);
    cudaFree(r);
    cudaFree(e);
    return s;
}

extern "C" nl_status nl_plan_set_net(nl_plan *p, nl_net *n)
{
    if (!nl_plan_ok(p) || (n && !net_ok(n))) {
        nl_set_error("nl_plan_set_net: bad argument");
        return NL_EINVAL;
    }
    p->net = n;
    return NL_OK;
}

extern "C" nl_status nl_net_set_coarse(nl_net *n, int block)
{
    if (!net_ok(n) || block < 0 || block == 1 || block > 65536) {
        nl_set_error("nl_net_set_coarse: bad argument (block 0 or 2 .. 65536)");
        return NL_EINVAL;
    }
    if (n->block != block) n->gen = next_generation();   // captured launch arguments change
    n->block = block;
    return NL_OK;
}
