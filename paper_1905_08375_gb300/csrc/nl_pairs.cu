// nl_pairs.cu -- the 2-D symmetric direct apply (Eq. (2.1)-(2.2), divergence form) for FP64
// data with arithmetic in pairs of FP32 numbers (NL_F64_PAIRS): the operator of the true
// residual f + L x that conjugate gradients checks at the end of its FP32 iterations.
//
// FP64 runs at 1/64 of the FP32 rate on this GPU, so the FP64 operator is the slowest launch
// of a solve.  Here every FP64 value v is carried as an unevaluated sum hi + lo of two FP32
// numbers (hi = fl32(v), lo = fl32(v - hi): 48 significant bits) and every step uses the
// error-free transformations of FP32 arithmetic (Knuth's TwoSum for the sum of two FP32
// numbers; the product of two FP32 numbers and its exact remainder by one fused
// multiply-add), as in double-word arithmetic (Dekker 1971; Joldes, Muller and Popescu,
// ACM TOMS 2017).  The term of output i at offset o (neighbour j),
//     g(o) b_j (w_i [o^2 <= thr_i] + w_j [o^2 <= thr_j]) (u_j - u_i),
// is split as w_i A_i + B_i with A_i = sum m_i g b_j d_ij and B_i = sum m_j g c_j d_ij,
// c_j = w_j b_j, d_ij = u_j - u_i; each term carries a relative error of a few 2^-46 of
// |g b_j d_ij| (the difference d_ij is formed exactly from the high words), the two
// accumulators are renormalised every 16 terms, and the epilogue
// b_i (w_i A_i + B_i - u_i ext_i) runs in FP64.  Explicitly rounded intrinsics keep the
// compiler from contracting the transformations.
//
// Layout: one thread per output, blocks of 32 x 8 outputs, a halo tile (32 + 2 RM) x
// (8 + 2 RM) staged in shared memory as six FP32 planes (u, b, c as hi | lo) and the
// thresholds + 1 (0 off the grid); the offset table sorted by |o|^2 holds the tile offset,
// |o|^2 and g(o) as hi | lo.  A warp walks the table up to the largest count of its outputs;
// the prefix in which every output's ball and every staged node's ball hold the offset skips
// the masks.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "nl_internal.cuh"

namespace {

constexpr int PB_X = 32, PB_Y = 8;       // outputs per block
constexpr int PAIR_RENORM = 16;          // terms between renormalisations of the accumulators

struct PairArgs {
    int n;
    int64_t N;
    const int *thr, *cnt;
    const float4 *bc;        // per node (b hi, b lo, c hi, c lo)
    const float4 *tab;       // per offset (tile offset bits, |o|^2 bits, g hi, g lo)
    int num_off;
    const double *wh, *fin, *ext;
};

// a + b = s + e exactly (Knuth's TwoSum; no condition on the magnitudes)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float ap = __fsub_rn(s, b);
    const float bp = __fsub_rn(s, ap);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// (xh + xl) (yh + yl) as ph + pl: ph = fl(xh yh), pl = its exact remainder plus the cross
// terms (the product xl yl, below 2^-48 of the result, is left out)
__device__ __forceinline__ void pair_mul(float xh, float xl, float yh, float yl, float &ph,
                                         float &pl)
{
    ph = __fmul_rn(xh, yh);
    float r = __fmaf_rn(xh, yh, -ph);
    r = __fmaf_rn(xh, yl, r);
    pl = __fmaf_rn(xl, yh, r);
}

// acc (hi, lo) += t (hi, lo): the high words by TwoSum, the low words and the rounding error
// added to the low accumulator
__device__ __forceinline__ void pair_acc(float &ah, float &al, float th, float tl)
{
    float s, e;
    two_sum(ah, th, s, e);
    ah = s;
    al = __fadd_rn(al, __fadd_rn(tl, e));
}

// the same sum with |al| at most half an ulp of ah (TwoSum of the two words)
__device__ __forceinline__ void pair_renorm(float &ah, float &al)
{
    float s, e;
    two_sum(ah, al, s, e);
    ah = s;
    al = e;
}

template <bool MASK>
__device__ __forceinline__ void pair_term(const float *__restrict__ sm, int PL, int q,
                                          float4 e, float uih, float uil, int ti, float &Ah,
                                          float &Al, float &Bh, float &Bl)
{
    const float ujh = sm[q], ujl = sm[q + PL];
    const float bh = sm[q + 2 * PL], bl = sm[q + 3 * PL];
    const float ch = sm[q + 4 * PL], cl = sm[q + 5 * PL];
    // d = u_j - u_i: the high words exactly by TwoSum, the low words added to the error
    float dh, de;
    two_sum(ujh, -uih, dh, de);
    const float dl = __fadd_rn(__fsub_rn(ujl, uil), de);
    // g d
    float gh, gl;
    pair_mul(e.z, e.w, dh, dl, gh, gl);
    float th, tl, vh, vl;
    pair_mul(bh, bl, gh, gl, th, tl);
    pair_mul(ch, cl, gh, gl, vh, vl);
    if (MASK) {
        const int o2 = __float_as_int(e.y);
        const int tj = reinterpret_cast<const int *>(sm)[q + 6 * PL];
        if (o2 >= ti) { th = 0.f; tl = 0.f; }
        if (o2 >= tj) { vh = 0.f; vl = 0.f; }
    }
    pair_acc(Ah, Al, th, tl);
    pair_acc(Bh, Bl, vh, vl);
}

template <int RM>
__global__ void __launch_bounds__(PB_X * PB_Y) k_sym2d_pairs(PairArgs a,
                                                            const double *__restrict__ u,
                                                            double *__restrict__ Lu)
{
    constexpr int SX = PB_X + 2 * RM, SY = PB_Y + 2 * RM, PL = SX * SY;
    extern __shared__ __align__(16) float sm[];          // uh | ul | bh | bl | ch | cl | thr + 1
    __shared__ int s_jmin[PB_Y];
    int *st = reinterpret_cast<int *>(sm) + 6 * PL;
    const int n = a.n;
    const int x0 = blockIdx.x * PB_X, y0 = blockIdx.y * PB_Y;
    const double *__restrict__ ur = u + (int64_t)blockIdx.z * a.N;
    const int tid = threadIdx.x + PB_X * threadIdx.y;
    int jmin = 0x7fffffff;                                // smallest thr + 1 of the staged nodes
    for (int e = tid; e < PL; e += PB_X * PB_Y) {
        const int gx = x0 - RM + e % SX, gy = y0 - RM + e / SX;
        float uh = 0.f, ul = 0.f;
        float4 bc = make_float4(0.f, 0.f, 0.f, 0.f);
        int t = 0;
        if (gx >= 0 && gx < n && gy >= 0 && gy < n) {
            const int64_t j = gx + (int64_t)n * gy;
            const double uv = ur[j];
            uh = __double2float_rn(uv);
            ul = __double2float_rn(uv - (double)uh);
            bc = a.bc[j];
            t = a.thr[j] + 1;
            jmin = min(jmin, t);
        }
        sm[e] = uh;
        sm[e + PL] = ul;
        sm[e + 2 * PL] = bc.x;
        sm[e + 3 * PL] = bc.y;
        sm[e + 4 * PL] = bc.z;
        sm[e + 5 * PL] = bc.w;
        st[e] = t;
    }
    jmin = __reduce_min_sync(0xffffffffu, jmin);
    if (threadIdx.x == 0) s_jmin[threadIdx.y] = jmin;
    __syncthreads();
#pragma unroll
    for (int w = 0; w < PB_Y; ++w) jmin = min(jmin, s_jmin[w]);

    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool act = x < n && y < n;
    const int64_t i = act ? x + (int64_t)n * y : 0;
    const int q0 = (threadIdx.y + RM) * SX + threadIdx.x + RM;
    const float uih = sm[q0], uil = sm[q0 + PL];
    const int ti = act ? a.thr[i] + 1 : 0x7fffffff;
    const int cnt_w = __reduce_max_sync(0xffffffffu, act ? a.cnt[i] : 0);
    const int tmin_w = __reduce_min_sync(0xffffffffu, ti);
    // offsets below both bounds hold every output's and every staged node's ball: no masks
    const int bound = min(jmin, tmin_w);
    int lo = 0, hi = cnt_w;
    while (lo < hi) {                                     // first entry with |o|^2 >= bound
        const int mid = (lo + hi) >> 1;
        if (__float_as_int(__ldg(&a.tab[mid]).y) < bound) lo = mid + 1; else hi = mid;
    }
    const int c_free = lo;
    float Ah = 0.f, Al = 0.f, Bh = 0.f, Bl = 0.f;
    int t = 0;
    while (t < c_free) {
        const int stop = min(c_free, t + PAIR_RENORM);
        for (; t < stop; ++t) {
            const float4 e = __ldg(&a.tab[t]);
            pair_term<false>(sm, PL, q0 + __float_as_int(e.x), e, uih, uil, ti, Ah, Al, Bh, Bl);
        }
        pair_renorm(Ah, Al);
        pair_renorm(Bh, Bl);
    }
    while (t < cnt_w) {
        const int stop = min(cnt_w, t + PAIR_RENORM);
        for (; t < stop; ++t) {
            const float4 e = __ldg(&a.tab[t]);
            pair_term<true>(sm, PL, q0 + __float_as_int(e.x), e, uih, uil, ti, Ah, Al, Bh, Bl);
        }
        pair_renorm(Ah, Al);
        pair_renorm(Bh, Bl);
    }
    if (!act) return;
    const double A = (double)Ah + (double)Al, B = (double)Bh + (double)Bl;
    const double ui = ur[i];
    Lu[(int64_t)blockIdx.z * a.N + i] = a.fin[i] * ((a.wh[i] * A + B) - ui * a.ext[i]);
}

// per node (b hi, b lo, c hi, c lo), c = w b
__global__ void k_pair_nodes(int64_t N, const double *__restrict__ b,
                             const double *__restrict__ wh, float4 *__restrict__ bc)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double bv = b[i], cv = wh[i] * bv;
    const float bh = __double2float_rn(bv), ch = __double2float_rn(cv);
    bc[i] = make_float4(bh, __double2float_rn(bv - (double)bh), ch,
                        __double2float_rn(cv - (double)ch));
}

template <int RM>
constexpr size_t pair_smem() { return sizeof(float) * 7 * (PB_X + 2 * RM) * (PB_Y + 2 * RM); }

template <int RM>
nl_status launch_pairs(const nl_plan *p, const PairArgs &a, const double *u, double *Lu,
                       int nrhs, cudaStream_t st)
{
    auto kern = k_sym2d_pairs<RM>;
    constexpr size_t smem = pair_smem<RM>();
    NL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    const dim3 grd((unsigned)((p->n + PB_X - 1) / PB_X), (unsigned)((p->n + PB_Y - 1) / PB_Y),
                   (unsigned)nrhs);
    kern<<<grd, dim3(PB_X, PB_Y, 1), smem, st>>>(a, u, Lu);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

float bits_as_float(int v)
{
    float f;
    std::memcpy(&f, &v, sizeof f);
    return f;
}

}  // namespace

// Plan set-up for NL_F64_PAIRS (2-D symmetric NL_POWER plans with Rmax <= 32): the halo of
// the tile, the offset table in the tile's geometry with g(o) split into hi | lo, and the
// per-node (b, c) pairs.  Other plans keep pair_rm = 0.
nl_status nl_pairs_plan_init(nl_plan *p, const int4 *offs, const double *g, int count,
                             cudaStream_t st)
{
    p->pair_rm = 0;
    if (p->d != 2 || !p->symmetric || p->family != NL_POWER || p->Rmax > 32 || count < 1)
        return NL_OK;
    const int rm = p->Rmax <= 4 ? 4 : p->Rmax <= 8 ? 8 : p->Rmax <= 16 ? 16 : p->Rmax <= 24 ? 24 : 32;
    const int SX = PB_X + 2 * rm;
    std::vector<float4> tab((size_t)count);
    for (int t = 0; t < count; ++t) {
        const int4 o = offs[t];
        const float gh = (float)g[t];
        tab[t] = make_float4(bits_as_float(o.x + SX * o.y), bits_as_float(o.w), gh,
                             (float)(g[t] - (double)gh));
    }
    float4 *dtab = nullptr, *dbc = nullptr;
    if (cudaMalloc(&dtab, tab.size() * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&dbc, (size_t)p->N * sizeof(float4)) != cudaSuccess) {
        if (dtab) cudaFree(dtab);
        nl_set_error("nl_plan_create: allocation of the FP32-pair tables failed");
        return NL_ENOMEM;
    }
    p->pair_tab = dtab;
    p->pair_bc = dbc;
    p->device_bytes += tab.size() * sizeof(float4) + (size_t)p->N * sizeof(float4);
    NL_CUDA_TRY(cudaMemcpyAsync(dtab, tab.data(), tab.size() * sizeof(float4),
                                cudaMemcpyHostToDevice, st));
    k_pair_nodes<<<(unsigned)((p->N + 255) / 256), 256, 0, st>>>(p->N, p->b64, p->wh64, dbc);
    NL_CUDA_TRY(cudaGetLastError());
    NL_CUDA_TRY(cudaStreamSynchronize(st));          // the host table is freed on return
    p->pair_rm = rm;
    return NL_OK;
}

nl_status nl_pairs_launch(const nl_plan *p, const double *u, double *Lu, int nrhs,
                          cudaStream_t st)
{
    if (!p->pair_rm) {
        nl_set_error("nl_apply: NL_F64_PAIRS is built for 2-D symmetric NL_POWER plans with "
                     "Rmax <= 32");
        return NL_EUNSUPPORTED;
    }
    PairArgs a;
    a.n = p->n; a.N = p->N;
    a.thr = p->thr; a.cnt = p->cnt;
    a.bc = p->pair_bc; a.tab = p->pair_tab; a.num_off = p->num_off;
    a.wh = p->wh64; a.fin = p->fin64; a.ext = p->ext64;
    switch (p->pair_rm) {
    case 4: return launch_pairs<4>(p, a, u, Lu, nrhs, st);
    case 8: return launch_pairs<8>(p, a, u, Lu, nrhs, st);
    case 16: return launch_pairs<16>(p, a, u, Lu, nrhs, st);
    case 24: return launch_pairs<24>(p, a, u, Lu, nrhs, st);
    default: return launch_pairs<32>(p, a, u, Lu, nrhs, st);
    }
}
