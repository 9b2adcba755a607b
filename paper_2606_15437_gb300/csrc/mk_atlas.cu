// mk_atlas.cu -- the failure-density atlas and its views (Sec. 9).
//
// atlas_kernel: D_ij's numerator, the number of (valuation, world) pairs
// at which formula i is false on frame j.  The frames are few (512 at three
// worlds) and the valuations many, so the layout is the census's turned
// around: a thread owns one frame (its n*n edges are uniform all-ones /
// all-zeros words) and the 32 lanes of a word are 32 consecutive
// valuations; atom p_i at world w is then a lane pattern (bit i*n+w of the
// valuation index), staged per valuation word as shared-memory rows, and a
// program step is the census interpreter unchanged.  The count is a
// popcount per world and valuation word.
//
// Seriation: column means and the centred Gram matrix G = Dc^T Dc in FP64
// (a tiled SIMT product), its leading eigenvectors by power iteration with
// deflation against earlier ones (one CTA), formula coordinates Dc v, and a
// bitonic sort of (coordinate, index) keys.  A(pi) is computed exactly as
// per-row integer sums of |count_i,pi(j+1) - count_i,pi(j)|.
//
// Density view: a 2-D histogram of points in FP64 cell arithmetic (integer
// atomics, so the counts are exact), and its occupancy statistics,
// including the pixels a square mark of radius r around each occupied cell
// would cover.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "mk.h"
#include "mk_attr.h"
#include "mk_eval.cuh"

namespace mkd {

constexpr int AT_BLOCK = 256;
constexpr int AT_U = 4;
constexpr int AT_ROW_CAP = 64;               // valuation words staged at a time
constexpr int AT_OPS_STRIDE = MK_MAX_CODE + 2;
constexpr int AT_TILE = 4;                  // formulas per CTA: short CTAs, a fuller grid

struct AtlasArgs {
    const mk_program *progs;
    int32_t nprog;
    uint64_t nframes;
    uint32_t *counts;
    uint64_t ld;
    int32_t *status;
};

template <int N, int U, int BLOCK>
struct AtlasSmem {
    static constexpr size_t code_bytes() { return ((size_t)AT_TILE * AT_OPS_STRIDE * 3 + 15) & ~(size_t)15; }
    static constexpr size_t meta_bytes() { return ((size_t)AT_TILE * 8 + 15) & ~(size_t)15; }
    static constexpr size_t row_bytes() { return (size_t)(AT_ROW_CAP + U) * RowShape<N>::WORDS * 4; }
    static constexpr size_t stack_bytes() { return (size_t)MK_MAX_STACK * U * N * BLOCK * 4; }
    static constexpr size_t total() { return code_bytes() + meta_bytes() + row_bytes() + stack_bytes(); }
};

// Word w of variable i in the atom row of valuation word q: lane l holds
// valuation 32q + l, so the word is bit i*N+w of that index across lanes.
template <int N>
__device__ __forceinline__ uint32_t lane_atom_word(uint32_t q, int idx) {
    const int i = idx / RowShape<N>::RS, w = idx % RowShape<N>::RS;
    if (w >= N) return 0u;
    const int b = i * N + w;
    return b < 5 ? lane_pattern(b) : bit_word((uint64_t)q << 5, b);
}

// Formulas whose valuations on n worlds number at most 8 (k*n <= 3, the
// variable-free and, at n = 2 or 3, the one-variable ones) would fill only
// 1-8 of a word's 32 valuation lanes; they are counted by
// atlas_packed_kernel instead, whose word holds 4 frames x 8 valuations.
template <int N>
__device__ __forceinline__ bool atlas_packed(int k) { return N >= 2 && k * N <= 3; }

template <int N, int U, int BLOCK>
__global__ void __launch_bounds__(BLOCK) atlas_kernel(AtlasArgs a) {
    using SM = AtlasSmem<N, U, BLOCK>;
    constexpr int RW = RowShape<N>::WORDS;
    extern __shared__ __align__(16) uint8_t smem[];
    uint16_t *s_offs = (uint16_t *)smem;
    uint8_t *s_ops = smem + (size_t)AT_TILE * AT_OPS_STRIDE * 2;
    int *s_nin = (int *)(smem + SM::code_bytes());
    int *s_k = s_nin + AT_TILE;
    uint32_t *s_rows = (uint32_t *)(smem + SM::code_bytes() + SM::meta_bytes());
    uint32_t *s_stack = (uint32_t *)((uint8_t *)s_rows + SM::row_bytes()) + threadIdx.x;

    const int p0 = blockIdx.y * AT_TILE;
    const int np = min(AT_TILE, a.nprog - p0);
    for (int i = threadIdx.x; i < np; i += BLOCK) {
        const mk_program &p = a.progs[p0 + i];
        int nin = -1;
        if (program_ok(p)) {
            nin = p.n_instr;
            if (p.nvars * N > 16) {
                nin = -1;
                if (blockIdx.x == 0) atomicOr(a.status, (int)MK_ST_LIMIT);
            } else if (atlas_packed<N>(p.nvars)) {
                nin = -1;                              // counted by atlas_packed_kernel
            }
        } else if (blockIdx.x == 0) {
            atomicOr(a.status, (int)MK_ST_PROGRAM);
        }
        s_nin[i] = nin;
        s_k[i] = p.nvars;
        if (nin >= 0) decode_program<N, U, BLOCK, false>(p, s_ops + i * AT_OPS_STRIDE, s_offs + i * AT_OPS_STRIDE);
    }
    __syncthreads();

    const uint64_t f = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
    uint32_t E[1][N * N];
#pragma unroll
    for (int e = 0; e < N * N; ++e) E[0][e] = f < a.nframes ? bit_word(f, e) : 0u;
    int rows_q0 = -1;
    for (int fi = 0; fi < np; ++fi) {
        if (s_nin[fi] < 0) continue;
        const uint32_t nval = 1u << (s_k[fi] * N);
        const uint32_t nq = (nval + 31) / 32;
        const uint8_t *ops = s_ops + fi * AT_OPS_STRIDE;
        const uint16_t *offs = s_offs + fi * AT_OPS_STRIDE;
        uint32_t cnt = 0;
        for (uint32_t q0 = 0; q0 < nq; q0 += AT_ROW_CAP) {
            if (rows_q0 != (int)q0) {
                __syncthreads();
                for (uint32_t i = threadIdx.x; i < AT_ROW_CAP * RW; i += BLOCK)
                    s_rows[i] = lane_atom_word<N>(q0 + i / RW, (int)(i % RW));
                __syncthreads();
                rows_q0 = (int)q0;
            }
            const uint32_t qn = min((uint32_t)AT_ROW_CAP, nq - q0);
            for (uint32_t qq = 0; qq < qn; qq += U) {
                uint32_t A[U][N];
                run_program<N, U, 1, BLOCK, RW, false>(ops, offs, s_rows + qq * RW, E, s_stack, A);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t q = q0 + qq + u;
                    uint32_t lanes = 0;
                    if (qq + u < qn) {
                        const uint32_t left = nval - 32 * q;
                        lanes = left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
                    }
#pragma unroll
                    for (int w = 0; w < N; ++w) cnt += __popc(~A[u][w] & lanes);
                }
            }
        }
        if (f < a.nframes) a.counts[(size_t)(p0 + fi) * a.ld + f] = cnt;
    }
}

// The counts of the formulas with at most 8 valuations per frame.  Lane l
// of word q holds frame 4q + (l >> 3) under valuation l & 7: frame-index
// bits 0 and 1 are lane bits 3 and 4 (lane patterns), the higher ones are
// the same for the whole word, and atom p_0 at world w is valuation bit w,
// a lane pattern too (k*n <= 3, so no valuation bit beyond bit 2).  One
// program run covers 4 frames under all their valuations; lanes of unused
// valuations are masked.  Needs N >= 2 (at least 4 frames).
template <int N, int BLOCK>
__global__ void __launch_bounds__(BLOCK) atlas_packed_kernel(AtlasArgs a) {
    constexpr int RW = RowShape<N>::WORDS;
    constexpr int RS = RowShape<N>::RS;
    __shared__ uint16_t s_offs[AT_TILE * AT_OPS_STRIDE];
    __shared__ uint8_t s_ops[AT_TILE * AT_OPS_STRIDE];
    __shared__ int s_nin[AT_TILE], s_k[AT_TILE];
    __shared__ __align__(16) uint32_t s_row[RW];
    extern __shared__ __align__(16) uint32_t s_pstack[];       // MK_MAX_STACK x N words per thread
    static_assert(N >= 2, "four frames per word");

    const int p0 = blockIdx.y * AT_TILE;
    const int np = min(AT_TILE, a.nprog - p0);
    for (int i = threadIdx.x; i < np; i += BLOCK) {
        const mk_program &p = a.progs[p0 + i];
        const int nin = program_ok(p) && atlas_packed<N>(p.nvars) ? p.n_instr : -1;
        s_nin[i] = nin;
        s_k[i] = p.nvars;
        if (nin >= 0) decode_program<N, 1, BLOCK, false>(p, s_ops + i * AT_OPS_STRIDE, s_offs + i * AT_OPS_STRIDE);
    }
    for (int i = threadIdx.x; i < RW; i += BLOCK) {
        const int v = i / RS, w = i % RS, b = v * N + w;
        s_row[i] = (w < N && b < 3) ? lane_pattern(b) : 0u;
    }
    __syncthreads();

    const uint64_t q = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;   // word: frames 4q .. 4q+3
    const uint64_t nwords = a.nframes / 4;
    uint32_t E[1][N * N];
#pragma unroll
    for (int e = 0; e < N * N; ++e) E[0][e] = e < 2 ? lane_pattern(3 + e) : bit_word(q << 2, e);
    if (q >= nwords) return;                                         // no barrier follows
    for (int fi = 0; fi < np; ++fi) {
        if (s_nin[fi] < 0) continue;
        const uint32_t nval = 1u << (s_k[fi] * N);                   // 1, 4 or 8
        const uint32_t vmask = nval >= 8 ? 0xFFFFFFFFu : 0x01010101u * ((1u << nval) - 1u);
        uint32_t A[1][N];
        run_program<N, 1, 1, BLOCK, 0, false>(s_ops + fi * AT_OPS_STRIDE, s_offs + fi * AT_OPS_STRIDE, s_row, E,
                                              s_pstack + threadIdx.x, A);
        uint32_t bad[N];
#pragma unroll
        for (int w = 0; w < N; ++w) bad[w] = ~A[0][w] & vmask;
        uint32_t *out = a.counts + (size_t)(p0 + fi) * a.ld + 4 * q;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            uint32_t c = 0;
#pragma unroll
            for (int w = 0; w < N; ++w) c += __popc(bad[w] & (0xFFu << (8 * g)));
            out[g] = c;
        }
    }
}

// Column means of D = counts / denom (one thread per column).
__global__ void colmean_kernel(const uint32_t *counts, const uint64_t *denom, int32_t B, int32_t F, uint64_t ld,
                               double *mean) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= F) return;
    double s = 0.0;
    for (int i = 0; i < B; ++i) s += (double)counts[(size_t)i * ld + j] / (double)denom[i];
    mean[j] = s / (double)B;
}

// G[a][b] = sum_i (D_ia - m_a)(D_ib - m_b): 32 x 32 output tiles, rows
// of D staged 32 at a time.
__global__ void gram_kernel(const uint32_t *counts, const uint64_t *denom, int32_t B, int32_t F, uint64_t ld,
                            const double *mean, double *G) {
    __shared__ double sa[32][33], sb[32][33];
    const int ta = blockIdx.y * 32, tb = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads, 4 outputs each
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i0 = 0; i0 < B; i0 += 32) {
        for (int r = ty; r < 32; r += 8) {
            const int i = i0 + r;
            double va = 0.0, vb = 0.0;
            if (i < B) {
                const double inv = 1.0 / (double)denom[i];
                if (ta + tx < F) va = (double)counts[(size_t)i * ld + ta + tx] * inv - mean[ta + tx];
                if (tb + tx < F) vb = (double)counts[(size_t)i * ld + tb + tx] * inv - mean[tb + tx];
            }
            sa[r][tx] = va;
            sb[r][tx] = vb;
        }
        __syncthreads();
        for (int r = 0; r < 32; ++r) {
            const double b = sb[r][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += sa[r][ty + 8 * q] * b;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = ta + ty + 8 * q, c = tb + tx;
        if (r < F && c < F) G[(size_t)r * F + c] = acc[q];
    }
}

// Leading eigenvector of the symmetric matrix G (F x F) orthogonal to the
// nprev vectors in prev (F each), by power iteration from a fixed start;
// one CTA, the iterate in shared memory, one warp per row of G (coalesced
// reads).  Stops after `iters` steps or once a step moves the unit vector
// by less than 1e-14 (squared distance 1e-28).  Sign: the largest-magnitude
// component is made positive.
__global__ void power_kernel(const double *G, int32_t F, const double *prev, int32_t nprev, int32_t iters,
                             double *v_out, double *lambda_out) {
    extern __shared__ __align__(16) double s_pw[];
    double *v = s_pw, *w = s_pw + F;
    __shared__ double red[32];
    __shared__ double s_val;
    const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, warp = t >> 5, nw = nt >> 5;
    auto block_sum = [&](double x) -> double {
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
        __syncthreads();
        if (lane == 0) red[warp] = x;
        __syncthreads();
        if (t < 32) {
            double y = t < nw ? red[t] : 0.0;
            for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xFFFFFFFFu, y, o);
            if (t == 0) s_val = y;
        }
        __syncthreads();
        return s_val;
    };
    for (int j = t; j < F; j += nt) v[j] = 1.0 + (double)j / (double)F;
    __syncthreads();
    double lam = 0.0;
    for (int it = 0; it < iters; ++it) {
        for (int p = 0; p < nprev; ++p) {      // deflate: v -= (v . q) q
            double d = 0.0;
            for (int j = t; j < F; j += nt) d += v[j] * prev[(size_t)p * F + j];
            d = block_sum(d);
            for (int j = t; j < F; j += nt) v[j] -= d * prev[(size_t)p * F + j];
            __syncthreads();
        }
        for (int r = warp; r < F; r += nw) {
            const double *row = G + (size_t)r * F;
            double s = 0.0;
            for (int j = lane; j < F; j += 32) s += row[j] * v[j];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
            if (lane == 0) w[r] = s;
        }
        __syncthreads();
        double nn = 0.0, vw = 0.0;
        for (int j = t; j < F; j += nt) {
            nn += w[j] * w[j];
            vw += v[j] * w[j];
        }
        nn = block_sum(nn);
        vw = block_sum(vw);
        lam = vw;
        const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
        double dd = 0.0;
        for (int j = t; j < F; j += nt) {
            const double x = w[j] * inv;
            dd += (x - v[j]) * (x - v[j]);
            v[j] = x;
        }
        dd = block_sum(dd);
        if (it >= 16 && dd < 1e-28) break;
    }
    // sign convention
    if (t == 0) {
        int best = 0;
        for (int j = 1; j < F; ++j)
            if (fabs(v[j]) > fabs(v[best])) best = j;
        s_val = v[best] < 0.0 ? -1.0 : 1.0;
        *lambda_out = lam;
    }
    __syncthreads();
    for (int j = t; j < F; j += nt) v_out[j] = v[j] * s_val;
}

// Formula coordinates u_i = sum_j (D_ij - m_j) v_j.
__global__ void project_kernel(const uint32_t *counts, const uint64_t *denom, int32_t B, int32_t F, uint64_t ld,
                               const double *mean, const double *v, double *u) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= B) return;
    const double inv = 1.0 / (double)denom[warp];
    double s = 0.0;
    for (int j = lane; j < F; j += 32) s += ((double)counts[(size_t)warp * ld + j] * inv - mean[j]) * v[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) u[warp] = s;
}

// Bitonic sort of (key, index) pairs ascending, ties by index.
__global__ void sort_init_kernel(const double *keys, int32_t n, int32_t P, double *k2, int32_t *idx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    k2[i] = i < n ? keys[i] : INFINITY;
    idx[i] = i;
}

__global__ void bitonic_kernel(double *k, int32_t *idx, int32_t P, int32_t size, int32_t stride) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const int j = i ^ stride;
    if (j <= i) return;
    const bool up = (i & size) == 0;
    const double ki = k[i], kj = k[j];
    const int ii = idx[i], ij = idx[j];
    const bool gt = ki > kj || (ki == kj && ii > ij);
    if (gt == up) {
        k[i] = kj;
        k[j] = ki;
        idx[i] = ij;
        idx[j] = ii;
    }
}

// Per-row integer sum of |count_i,perm(j+1) - count_i,perm(j)|.
__global__ void adjvar_kernel(const uint32_t *counts, int32_t B, int32_t F, uint64_t ld, const int32_t *perm,
                              uint64_t *rowsum, int32_t *status) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= B) return;
    const uint32_t *row = counts + (size_t)warp * ld;
    unsigned long long s = 0;
    for (int j = lane; j + 1 < F; j += 32) {
        const int32_t a = perm[j], b = perm[j + 1];
        if (a < 0 || a >= F || b < 0 || b >= F) {
            atomicOr(status, (int)MK_ST_INDEX);
            continue;
        }
        const int64_t d = (int64_t)row[b] - (int64_t)row[a];
        s += (unsigned long long)(d < 0 ? -d : d);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) rowsum[warp] = s;
}

__device__ __forceinline__ int cell_of(double z, double lo, double hi, int G) {
    double c = floor((z - lo) / (hi - lo) * (double)G);
    if (!(c >= 0.0)) c = 0.0;                  // also NaN
    if (c > (double)(G - 1)) c = (double)(G - 1);
    return (int)c;
}

__global__ void hist2d_kernel(const double *x, const double *y, int64_t npts, double lo, double hi, int32_t G,
                              uint32_t *hist) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npts; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[(size_t)cell_of(y[i], lo, hi, G) * G + cell_of(x[i], lo, hi, G)], 1u);
}

// stats: [0] occupied cells, [1] largest cell, [2] points in cells shared
// with another point, [3] pixels within Chebyshev distance r of an
// occupied cell.
__global__ void hist_stats_kernel(const uint32_t *hist, int32_t G, int32_t r, unsigned long long *stats) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= (int64_t)G * G) return;
    const uint32_t h = hist[c];
    if (h) {
        atomicAdd(&stats[0], 1ull);
        atomicMax(&stats[1], (unsigned long long)h);
        if (h > 1) atomicAdd(&stats[2], (unsigned long long)h);
    }
    const int cy = (int)(c / G), cx = (int)(c % G);
    bool cov = false;
    for (int dy = -r; dy <= r && !cov; ++dy)
        for (int dx = -r; dx <= r && !cov; ++dx) {
            const int yy = cy + dy, xx = cx + dx;
            if (yy >= 0 && yy < G && xx >= 0 && xx < G && hist[(size_t)yy * G + xx]) cov = true;
        }
    if (cov) atomicAdd(&stats[3], 1ull);
}

__global__ void zero_u64_kernel(unsigned long long *p, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0;
}

}  // namespace mkd

namespace {

using namespace mkd;


template <int N>
void launch_atlas(const AtlasArgs &a, cudaStream_t s) {
    using SM = AtlasSmem<N, AT_U, AT_BLOCK>;
    auto kern = atlas_kernel<N, AT_U, AT_BLOCK>;
    ensure_dynamic_smem((const void *)kern, SM::total());
    dim3 grid((unsigned)((a.nframes + AT_BLOCK - 1) / AT_BLOCK), (unsigned)((a.nprog + AT_TILE - 1) / AT_TILE));
    kern<<<grid, AT_BLOCK, SM::total(), s>>>(a);
    if constexpr (N >= 2) {
        constexpr int PB = 128;
        const uint64_t nwords = a.nframes / 4;
        const size_t stack = (size_t)MK_MAX_STACK * N * PB * 4;
        auto pk = atlas_packed_kernel<N, PB>;
        ensure_dynamic_smem((const void *)pk, stack);
        dim3 pgrid((unsigned)((nwords + PB - 1) / PB), (unsigned)((a.nprog + AT_TILE - 1) / AT_TILE));
        pk<<<pgrid, PB, stack, s>>>(a);
    }
}

int32_t pow2_at_least(int32_t n) {
    int32_t p = 1;
    while (p < n) p <<= 1;
    return p;
}

}  // namespace

extern "C" int mk_atlas_counts(const mk_program *d_progs, int32_t nprog, int32_t n, uint32_t *d_counts,
                               uint64_t ld, int32_t *d_status, void *stream) {
    if (n < 1 || n > 4 || nprog < 0 || !d_status) return MK_E_ARG;
    const uint64_t nf = 1ull << (n * n);
    if (ld < nf) return MK_E_ARG;
    if (nprog == 0) return MK_OK;
    if (!d_progs || !d_counts || (nprog + AT_TILE - 1) / AT_TILE > 65535) return MK_E_ARG;
    AtlasArgs a;
    std::memset(&a, 0, sizeof(a));
    a.progs = d_progs;
    a.nprog = nprog;
    a.nframes = nf;
    a.counts = d_counts;
    a.ld = ld;
    a.status = d_status;
    cudaStream_t s = (cudaStream_t)stream;
    switch (n) {
    case 1: launch_atlas<1>(a, s); break;
    case 2: launch_atlas<2>(a, s); break;
    case 3: launch_atlas<3>(a, s); break;
    case 4: launch_atlas<4>(a, s); break;
    }
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

extern "C" int mk_atlas_gram(const uint32_t *d_counts, const uint64_t *d_denom, int32_t B, int32_t F, uint64_t ld,
                             double *d_mean, double *d_gram, void *stream) {
    if (B < 1 || F < 1 || F > MK_MAX_ATLAS_AXIS || ld < (uint64_t)F || !d_counts || !d_denom || !d_mean || !d_gram)
        return MK_E_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    colmean_kernel<<<(F + 255) / 256, 256, 0, s>>>(d_counts, d_denom, B, F, ld, d_mean);
    dim3 grid((F + 31) / 32, (F + 31) / 32);
    gram_kernel<<<grid, 256, 0, s>>>(d_counts, d_denom, B, F, ld, d_mean, d_gram);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

extern "C" size_t mk_power_workspace_size(int32_t F) { return F > 0 ? (size_t)2 * F * sizeof(double) : 0; }

extern "C" int mk_power_iteration(const double *d_gram, int32_t F, const double *d_prev, int32_t nprev, int32_t iters,
                                  double *d_v, double *d_lambda, void *d_workspace, size_t ws_bytes, void *stream) {
    (void)d_workspace;
    (void)ws_bytes;
    if (F < 1 || F > MK_MAX_ATLAS_AXIS || nprev < 0 || iters < 1 || !d_gram || !d_v || !d_lambda || (nprev && !d_prev))
        return MK_E_ARG;
    const size_t sm = 2 * (size_t)F * sizeof(double);
    ensure_dynamic_smem((const void *)power_kernel, 2 * MK_MAX_ATLAS_AXIS * sizeof(double));
    power_kernel<<<1, 1024, sm, (cudaStream_t)stream>>>(d_gram, F, d_prev, nprev, iters, d_v, d_lambda);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

extern "C" int mk_atlas_project(const uint32_t *d_counts, const uint64_t *d_denom, int32_t B, int32_t F, uint64_t ld,
                                const double *d_mean, const double *d_v, double *d_u, void *stream) {
    if (B < 1 || F < 1 || ld < (uint64_t)F || !d_counts || !d_denom || !d_mean || !d_v || !d_u) return MK_E_ARG;
    const int64_t threads = (int64_t)B * 32;
    project_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_counts, d_denom, B, F, ld,
                                                                                       d_mean, d_v, d_u);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

extern "C" size_t mk_sort_workspace_size(int32_t n) {
    if (n < 1) return 0;
    const size_t P = (size_t)pow2_at_least(n);
    return P * (sizeof(double) + sizeof(int32_t));
}

extern "C" int mk_sort_keys(const double *d_keys, int32_t n, int32_t *d_order, void *d_workspace, size_t ws_bytes,
                            void *stream) {
    if (n < 1 || n > (1 << 30) || !d_keys || !d_order) return MK_E_ARG;
    if (!d_workspace || ws_bytes < mk_sort_workspace_size(n)) return MK_E_WORKSPACE;
    const int32_t P = pow2_at_least(n);
    double *k = (double *)d_workspace;
    int32_t *idx = (int32_t *)(k + P);
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned grid = (unsigned)((P + 255) / 256);
    sort_init_kernel<<<grid, 256, 0, s>>>(d_keys, n, P, k, idx);
    for (int32_t size = 2; size <= P; size <<= 1)
        for (int32_t stride = size >> 1; stride > 0; stride >>= 1) bitonic_kernel<<<grid, 256, 0, s>>>(k, idx, P, size, stride);
    cudaMemcpyAsync(d_order, idx, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

extern "C" int mk_adjacent_variation(const uint32_t *d_counts, int32_t B, int32_t F, uint64_t ld,
                                     const int32_t *d_perm, uint64_t *d_rowsum, int32_t *d_status, void *stream) {
    if (B < 1 || F < 2 || ld < (uint64_t)F || !d_counts || !d_perm || !d_rowsum || !d_status) return MK_E_ARG;
    const int64_t threads = (int64_t)B * 32;
    adjvar_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_counts, B, F, ld, d_perm,
                                                                                       d_rowsum, d_status);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

extern "C" int mk_histogram2d(const double *d_x, const double *d_y, int64_t npts, double lo, double hi, int32_t G,
                              uint32_t *d_hist, void *stream) {
    if (npts < 0 || G < 1 || G > 16384 || !(hi > lo) || (npts && (!d_x || !d_y)) || !d_hist) return MK_E_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(d_hist, 0, (size_t)G * G * sizeof(uint32_t), s);
    if (npts) hist2d_kernel<<<4 * 152, 256, 0, s>>>(d_x, d_y, npts, lo, hi, G, d_hist);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

extern "C" int mk_histogram_stats(const uint32_t *d_hist, int32_t G, int32_t radius, uint64_t *d_stats, void *stream) {
    if (G < 1 || G > 16384 || radius < 0 || radius > 16 || !d_hist || !d_stats) return MK_E_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    zero_u64_kernel<<<1, 32, 0, s>>>((unsigned long long *)d_stats, 4);
    const int64_t cells = (int64_t)G * G;
    hist_stats_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(d_hist, G, radius, (unsigned long long *)d_stats);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}
