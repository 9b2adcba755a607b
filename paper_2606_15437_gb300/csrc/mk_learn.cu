// mk_learn.cu -- the learned pair proposal: truth vectors, Hamming k-NN
// universe, and the MLP's training and inference kernels.
//
// The paper ranks candidate pairs by small-frame semantic representations
// (Sec. 9: fingerprints over frames and valuations, layouts, neighbour
// universes, exact verification of every hit).  Here the representation is
// a truth vector -- formula phi's truth value at each of M seeded pointed
// models -- and a small MLP learns, from pairs the exact search has
// labelled, which pairs are likely to agree on every small frame yet split
// on a larger one.  The exact separation search stays the only judge.
//
//   fingerprint_kernel<N>  bit j of phi's vector = M_j, w_j |= phi, for 32
//                          models of N worlds per thread (bit-sliced like the
//                          census, but every lane has its own frame and
//                          valuation, so atoms are per-lane words)
//   knn_kernel             exact k nearest neighbours in Hamming distance
//                          (distance histogram -> threshold -> ordered pick)
//   gemm kernels           FP32 tiled GEMM (training) whose first-layer
//                          operand is generated from the two truth vectors
//                          of each pair: x = [a xor b, a and b]
//   infer kernel           BF16 tensor-core (mma.sync m16n8k16) first layer
//                          for scoring large universes, FP32 accumulation
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "mk.h"
#include "mk_attr.h"
#include "mk_eval.cuh"

namespace mkd {

// ------------------------------------------------------------ truth vectors

// One thread = one group of 32 models of N worlds; the CTA walks a tile of
// formulas, so every thread runs the same program (uniform dispatch).
template <int N>
__global__ void __launch_bounds__(128) fingerprint_kernel(const mk_program *progs, int32_t nprog,
                                                          const mk_model *models, int32_t g0, int32_t ngroups,
                                                          int32_t words_per_vec, uint32_t *bits,
                                                          int32_t *status) {
    constexpr int RW = RowShape<N>::WORDS;
    constexpr int BLOCK = 128;
    __shared__ __align__(16) uint32_t s_rows[BLOCK * RW];
    __shared__ uint32_t s_stack[MK_MAX_STACK * N * BLOCK];
    __shared__ uint8_t s_ops[MK_MAX_CODE + 2];
    __shared__ uint16_t s_offs[MK_MAX_CODE + 2];
    __shared__ int s_ok;

    const int g = g0 + blockIdx.x * BLOCK + threadIdx.x;     // model group (global index)
    const bool active = g < g0 + ngroups;
    uint32_t E[1][N * N];
#pragma unroll
    for (int e = 0; e < N * N; ++e) E[0][e] = 0;
    uint32_t wm[N];                 // lanes whose pointed world is w
#pragma unroll
    for (int w = 0; w < N; ++w) wm[w] = 0;
    uint32_t *row = s_rows + threadIdx.x * RW;
#pragma unroll
    for (int i = 0; i < RW; ++i) row[i] = 0;
    if (active) {
        const mk_model *m = models + (size_t)g * 32;
        for (int l = 0; l < 32; ++l) {
            const uint64_t f = m[l].frame;
            const uint32_t v = m[l].val;
#pragma unroll
            for (int e = 0; e < N * N; ++e) E[0][e] |= (uint32_t)((f >> e) & 1u) << l;
#pragma unroll
            for (int i = 0; i < MK_MAX_VARS; ++i)
#pragma unroll
                for (int w = 0; w < N; ++w) row[i * RowShape<N>::RS + w] |= ((v >> (i * N + w)) & 1u) << l;
#pragma unroll
            for (int w = 0; w < N; ++w) wm[w] |= (uint32_t)(m[l].world == w) << l;
        }
    }
    const int p0 = blockIdx.y * 64;
    const int np = min(64, nprog - p0);
    for (int fi = 0; fi < np; ++fi) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const mk_program &p = progs[p0 + fi];
            s_ok = program_ok(p);
            if (s_ok) decode_program<N, 1, BLOCK>(p, s_ops, s_offs);
            else atomicOr(status, (int)MK_ST_PROGRAM);
        }
        __syncthreads();
        if (!s_ok) continue;
        uint32_t A[1][N];
        run_program<N, 1, 1, BLOCK, 0>(s_ops, s_offs, row, E, s_stack + threadIdx.x, A);
        uint32_t t = 0;
#pragma unroll
        for (int w = 0; w < N; ++w) t |= A[0][w] & wm[w];
        if (active) bits[(size_t)(p0 + fi) * words_per_vec + g] = t;
    }
}

// ------------------------------------------------------------ k-NN

// One CTA per query vector: Hamming distances to every vector (self
// excluded), a distance histogram, the threshold distance t with
// #(d < t) < k <= #(d <= t), then the neighbours: all with d < t and the
// lowest-index ones with d == t, in index order.
__global__ void __launch_bounds__(512) knn_kernel(const uint32_t *bits, int32_t nvec, int32_t words, int32_t k,
                                                  int32_t *nbr, uint16_t *dist_out, uint16_t *dist_scratch) {
    extern __shared__ uint32_t s_hist[];      // words + 1 bins of the histogram, then the query
    const int q = blockIdx.x;
    const int nb = words * 32 + 1;
    uint32_t *s_q = s_hist + nb;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s_hist[i] = 0;
    for (int i = threadIdx.x; i < words; i += blockDim.x) s_q[i] = bits[(size_t)q * words + i];
    __syncthreads();
    uint16_t *d = dist_scratch + (size_t)q * nvec;
    for (int j = threadIdx.x; j < nvec; j += blockDim.x) {
        uint32_t s = 0;
        const uint32_t *v = bits + (size_t)j * words;
        for (int i = 0; i < words; ++i) s += __popc(v[i] ^ s_q[i]);
        d[j] = (uint16_t)s;
        if (j != q) atomicAdd(&s_hist[s], 1u);
    }
    __syncthreads();
    __shared__ int s_t, s_below;
    if (threadIdx.x == 0) {
        int acc = 0, t = nb;     // nb: fewer than k others, all of them are neighbours
        for (int b = 0; b < nb; ++b) {
            if (acc + (int)s_hist[b] >= k) { t = b; break; }
            acc += (int)s_hist[b];
        }
        s_t = t;
        s_below = acc;
    }
    __syncthreads();
    const int t = s_t;
    const int kk = min(k, nvec - 1);
    // ordered pick: warp ballots over index blocks, one warp at a time in order
    __shared__ int s_lo, s_eq;
    if (threadIdx.x == 0) { s_lo = 0; s_eq = 0; }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int base = 0; base < nvec; base += blockDim.x) {
        const int j = base + threadIdx.x;
        const uint16_t dj = j < nvec ? d[j] : 0xFFFF;
        const bool lt = j < nvec && j != q && dj < t;
        const bool eq = j < nvec && j != q && dj == t;
        // rank within the block, warp by warp
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
            if ((int)(threadIdx.x >> 5) == w) {
                const uint32_t blt = __ballot_sync(0xFFFFFFFFu, lt), beq = __ballot_sync(0xFFFFFFFFu, eq);
                const uint32_t below = (1u << lane) - 1u;
                if (lt) {
                    const int pos = s_lo + __popc(blt & below);
                    nbr[(size_t)q * k + pos] = j;
                    dist_out[(size_t)q * k + pos] = dj;
                }
                if (eq) {
                    const int r = s_eq + __popc(beq & below);
                    if (s_below + r < kk) {
                        nbr[(size_t)q * k + s_below + r] = j;
                        dist_out[(size_t)q * k + s_below + r] = dj;
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    s_lo += __popc(blt);
                    s_eq += __popc(beq);
                }
            }
            __syncthreads();
        }
    }
    for (int i = kk + threadIdx.x; i < k; i += blockDim.x) {
        nbr[(size_t)q * k + i] = -1;
        dist_out[(size_t)q * k + i] = 0xFFFF;
    }
}

// ------------------------------------------------------------ FP32 GEMM
//
// C[M x N] = op(A) * op(B) (+ bias, ReLU), 128 x 128 tiles, 8-deep k steps,
// 256 threads with 8 x 8 outputs each.  op(A) is read through a loader so
// the first layer's operand can be generated from truth vectors.

constexpr int GBM = 128, GBN = 128, GBK = 8;
constexpr int kGemmFill = 2 * 152;       // CTAs that fill a GB300 (two per SM)
constexpr int kGemmMinChunk = 256;       // least K per split-K chunk

enum { A_ROW = 0, A_COL = 1, A_PAIR = 2, A_PAIR_T = 3 };
enum { B_ROW = 0, B_COL = 1 };

struct GemmArgs {
    int32_t M, N, K;
    const float *A;            // A_ROW: A[m*lda + k]; A_COL: A[k*lda + m]
    int32_t lda;
    const uint32_t *vec;       // A_PAIR: truth vectors, words_per_vec words each
    const int32_t *pa, *pb;    //   pair p = (vec[pa[p]], vec[pb[p]])
    int32_t vwords;            //   feature f < 32*vwords: (a xor b) bit f, else (a and b)
    const float *B;            // B_ROW: B[k*ldb + n]; B_COL: B[n*ldb + k]
    int32_t ldb;
    float *C;
    int32_t ldc;
    const float *bias;         // per column, may be NULL
    int32_t relu;
    float beta;                // C = acc + beta * C
    int32_t kchunk;            // split K: CTA z takes k in [z*kchunk, (z+1)*kchunk) (0 = all of K)
    float *part;               //   and writes its raw sums to part[z][M][N] (the epilogue is later)
};

template <int AMODE>
__device__ __forceinline__ float load_a(const GemmArgs &g, int m, int k) {
    if (m >= g.M || k >= g.K) return 0.f;
    if constexpr (AMODE == A_ROW) return g.A[(size_t)m * g.lda + k];
    else if constexpr (AMODE == A_COL) return g.A[(size_t)k * g.lda + m];
    else {
        const int p = AMODE == A_PAIR ? m : k;       // pair
        const int f = AMODE == A_PAIR ? k : m;       // feature
        const int half = g.vwords * 32;
        const int fb = f < half ? f : f - half;
        const uint32_t a = g.vec[(size_t)g.pa[p] * g.vwords + (fb >> 5)];
        const uint32_t b = g.vec[(size_t)g.pb[p] * g.vwords + (fb >> 5)];
        const uint32_t x = f < half ? (a ^ b) : (a & b);
        return (float)((x >> (fb & 31)) & 1u);
    }
}

template <int BMODE>
__device__ __forceinline__ float load_b(const GemmArgs &g, int k, int n) {
    if (k >= g.K || n >= g.N) return 0.f;
    if constexpr (BMODE == B_ROW) return g.B[(size_t)k * g.ldb + n];
    else return g.B[(size_t)n * g.ldb + k];
}

// A thread's 8 x 8 outputs at (mb, nb): the raw sums into the split-K
// partials, or C = acc + beta * C + bias, then the ReLU.
__device__ __forceinline__ void gemm_store(const GemmArgs &g, const float (&acc)[8][8], int mb, int nb) {
    if (g.part) {
        float *pz = g.part + (size_t)blockIdx.z * g.M * g.N;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int m = mb + i;
            if (m >= g.M) continue;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (nb + j < g.N) pz[(size_t)m * g.N + nb + j] = acc[i][j];
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = mb + i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = nb + j;
            if (n >= g.N) continue;
            float v = acc[i][j];
            if (g.beta != 0.f) v += g.beta * g.C[(size_t)m * g.ldc + n];
            if (g.bias) v += g.bias[n];
            if (g.relu) v = v > 0.f ? v : 0.f;
            g.C[(size_t)m * g.ldc + n] = v;
        }
    }
}

template <int AMODE, int BMODE>
__global__ void __launch_bounds__(256) gemm_f32_kernel(GemmArgs g) {
    __shared__ float As[GBK][GBM + 4];
    __shared__ float Bs[GBK][GBN + 4];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int tm = (tid / 16) * 8, tn = (tid % 16) * 8;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    const int kb = g.kchunk ? (int)blockIdx.z * g.kchunk : 0;
    const int ke = g.kchunk ? min(g.K, kb + g.kchunk) : g.K;
    for (int k0 = kb; k0 < ke; k0 += GBK) {
        // 1024 elements of each tile, 4 per thread
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + r * 256;
            const int am = e % GBM, ak = e / GBM;
            As[ak][am] = k0 + ak < ke ? load_a<AMODE>(g, m0 + am, k0 + ak) : 0.f;
            const int bn = e % GBN, bk = e / GBN;
            Bs[bk][bn] = k0 + bk < ke ? load_b<BMODE>(g, k0 + bk, n0 + bn) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            float a[8], b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = As[kk][tm + i];
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] = Bs[kk][tn + j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    gemm_store(g, acc, m0 + tm, n0 + tn);
}

// The two GEMMs whose A operand is the pair features x = [a xor b, a and b]
// (forward x W1: rows = pairs, k = features; dW1 = x^T d1: rows = features,
// k = pairs), with 32-deep k steps: a truth-vector word holds 32 features,
// so each word is loaded once per tile row and expanded bit by bit into
// shared memory.  B is row-major [K][N].  Features f < F/2 take the xor of
// word f/32 of the two vectors, the others the and of word f/32 - F/64;
// F is a multiple of 64, so no 32-feature group straddles the two halves.
//
// Both operand tiles are double-buffered.  After the barrier that opens k
// step t, the CTA starts the B copies of step t+1 (cp.async, 16 bytes each,
// zero-filled past K) into the buffer step t-1 used, and loads the truth-
// vector words of step t+1 into registers (the transposed GEMM also the pair
// indices of step t+2); it then runs step t's FMAs and only afterwards
// expands those words into the other A buffer.  One barrier per k step
// separates the buffers, and the global loads run under the arithmetic.
constexpr int PBK = 32;
constexpr int PAIR_AS = PBK * (GBM + 4), PAIR_BS = PBK * (GBN + 4);   // floats per buffer
constexpr size_t kPairSmem = 2 * (size_t)(PAIR_AS + PAIR_BS) * sizeof(float);

__device__ __forceinline__ void pair_cp16(uint32_t dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void pair_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void pair_cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// B rows [k0, k0 + 32) x columns [n0, n0 + 128) into one buffer: by cp.async
// when every column exists and rows are 16-byte aligned, else by plain loads.
__device__ __forceinline__ void pair_load_b(const GemmArgs &g, float *bs, int k0, int ke, int n0, bool basync) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int e = tid + r * 256;                   // float4 index in the 32 x 32 float4 tile
        const int bk = e >> 5, bn = (e & 31) * 4;
        float *dst = bs + bk * (GBN + 4) + bn;
        if (basync) {
            const bool in = k0 + bk < ke;
            const float *src = in ? g.B + (size_t)(k0 + bk) * g.ldb + n0 + bn : g.B;
            pair_cp16((uint32_t)__cvta_generic_to_shared(dst), src, in ? 16u : 0u);
        } else {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k0 + bk < ke) {
                const float *row = g.B + (size_t)(k0 + bk) * g.ldb + n0 + bn;
                if (n0 + bn < g.N) v.x = row[0];
                if (n0 + bn + 1 < g.N) v.y = row[1];
                if (n0 + bn + 2 < g.N) v.z = row[2];
                if (n0 + bn + 3 < g.N) v.w = row[3];
            }
            *reinterpret_cast<float4 *>(dst) = v;
        }
    }
    if (basync) pair_cp_commit();
}

template <bool TRANS>
__global__ void __launch_bounds__(256, 2) gemm_pair_kernel(GemmArgs g) {
    extern __shared__ __align__(16) float pair_smem[];
    float *const As = pair_smem;                      // [2][PBK][GBM + 4]
    float *const Bs = pair_smem + 2 * PAIR_AS;        // [2][PBK][GBN + 4]
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int tm = (tid / 16) * 8, tn = (tid % 16) * 8;
    const int F = g.vwords * 64, halfF = g.vwords * 32;
    const bool basync = (g.ldb & 3) == 0 && ((uintptr_t)g.B & 15) == 0 && n0 + GBN <= g.N;
    const int kb = g.kchunk ? (int)blockIdx.z * g.kchunk : 0;
    const int ke = g.kchunk ? min(g.K, kb + g.kchunk) : g.K;
    const int nt = ke > kb ? (ke - kb + PBK - 1) / PBK : 0;

    // forward: thread t < 128 owns pair m0 + t for the whole K loop
    int ia = 0, ib = 0;
    bool prow = false;
    // transposed: thread (pair row tk of the step, sixteenth tj of the features)
    const int tk = tid >> 3, tj = tid & 7;
    const int f0 = m0 + tj * 16;
    const bool fcol = f0 < F;
    const int fw = (f0 < halfF ? f0 : f0 - halfF) >> 5;
    int nja = 0, njb = 0;                             // pair indices of the next step's row
    if constexpr (!TRANS) {
        if (tid < GBM && m0 + tid < g.M) {
            ia = g.pa[m0 + tid];
            ib = g.pb[m0 + tid];
            prow = true;
        }
    }

    // A words of the step at k0: forward, word k0/32 of this thread's pair;
    // transposed, word f0/32 of pair (ja, jb) (valid rows only)
    auto expand = [&](float *as, int k0, uint32_t a, uint32_t b) {
        if constexpr (!TRANS) {
            if (tid < GBM) {
                const uint32_t x = k0 < halfF ? (a ^ b) : (a & b);
#pragma unroll
                for (int kk = 0; kk < PBK; ++kk)
                    as[kk * (GBM + 4) + tid] = (k0 + kk < ke) ? (float)((x >> kk) & 1u) : 0.f;
            }
        } else {
            const uint32_t x = (f0 < halfF ? (a ^ b) : (a & b)) >> (f0 & 16);
#pragma unroll
            for (int i = 0; i < 16; ++i) as[tk * (GBM + 4) + tj * 16 + i] = (float)((x >> i) & 1u);
        }
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    // prologue: step 0 into buffer 0; the transposed GEMM's indices of step 1
    if (nt > 0) {
        pair_load_b(g, Bs, kb, ke, n0, basync);
        uint32_t a = 0, b = 0;
        if constexpr (!TRANS) {
            if (prow) {
                const int w = (kb < halfF ? kb : kb - halfF) >> 5;
                a = g.vec[(size_t)ia * g.vwords + w];
                b = g.vec[(size_t)ib * g.vwords + w];
            }
        } else {
            if (kb + tk < ke && fcol) {
                const int ja = g.pa[kb + tk], jb = g.pb[kb + tk];
                a = g.vec[(size_t)ja * g.vwords + fw];
                b = g.vec[(size_t)jb * g.vwords + fw];
            }
            if (nt > 1 && kb + PBK + tk < ke && fcol) {
                nja = g.pa[kb + PBK + tk];
                njb = g.pb[kb + PBK + tk];
            }
        }
        expand(As, kb, a, b);
    }

    for (int t = 0; t < nt; ++t) {
        const int k0 = kb + t * PBK;
        const float *as = As + (t & 1) * PAIR_AS, *bs = Bs + (t & 1) * PAIR_BS;
        float *as_next = As + ((t + 1) & 1) * PAIR_AS, *bs_next = Bs + ((t + 1) & 1) * PAIR_BS;
        if (basync) pair_cp_wait_all();
        __syncthreads();                               // step t's tiles are in; step t-1's reads are done
        const bool more = t + 1 < nt;
        const int k1 = k0 + PBK;
        uint32_t a = 0, b = 0;                         // step t+1's words
        if (more) {
            pair_load_b(g, bs_next, k1, ke, n0, basync);
            if constexpr (!TRANS) {
                if (prow) {
                    const int w = (k1 < halfF ? k1 : k1 - halfF) >> 5;
                    a = g.vec[(size_t)ia * g.vwords + w];
                    b = g.vec[(size_t)ib * g.vwords + w];
                }
            } else {
                if (k1 + tk < ke && fcol) {
                    a = g.vec[(size_t)nja * g.vwords + fw];
                    b = g.vec[(size_t)njb * g.vwords + fw];
                }
                if (t + 2 < nt && k1 + PBK + tk < ke && fcol) {
                    nja = g.pa[k1 + PBK + tk];
                    njb = g.pb[k1 + PBK + tk];
                }
            }
        }
#pragma unroll 8
        for (int kk = 0; kk < PBK; ++kk) {
            float av[8], bv[8];
            const float4 a0 = *reinterpret_cast<const float4 *>(as + kk * (GBM + 4) + tm);
            const float4 a1 = *reinterpret_cast<const float4 *>(as + kk * (GBM + 4) + tm + 4);
            const float4 b0 = *reinterpret_cast<const float4 *>(bs + kk * (GBN + 4) + tn);
            const float4 b1 = *reinterpret_cast<const float4 *>(bs + kk * (GBN + 4) + tn + 4);
            av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w;
            av[4] = a1.x; av[5] = a1.y; av[6] = a1.z; av[7] = a1.w;
            bv[0] = b0.x; bv[1] = b0.y; bv[2] = b0.z; bv[3] = b0.w;
            bv[4] = b1.x; bv[5] = b1.y; bv[6] = b1.z; bv[7] = b1.w;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (more) expand(as_next, k1, a, b);
    }
    if (basync) pair_cp_wait_all();
    gemm_store(g, acc, m0 + tm, n0 + tn);
}

// Split-K epilogue: C = sum_z part[z] (z in order, so the result does not
// depend on scheduling) + beta * C + bias, then the ReLU.
__global__ void splitk_epilogue_kernel(const float *part, int32_t S, int32_t M, int32_t N, float *C, int32_t ldc,
                                       const float *bias, int32_t relu, float beta) {
    const size_t mn = (size_t)M * N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < mn; i += (size_t)gridDim.x * blockDim.x) {
        float v = 0.f;
        for (int z = 0; z < S; ++z) v += part[(size_t)z * mn + i];
        const int m = (int)(i / N), n = (int)(i % N);
        if (beta != 0.f) v += beta * C[(size_t)m * ldc + n];
        if (bias) v += bias[n];
        if (relu) v = v > 0.f ? v : 0.f;
        C[(size_t)m * ldc + n] = v;
    }
}

// ------------------------------------------------------------ MLP pieces

// z[p] = h2[p] . w3 + b3; loss gradient dz[p] = w_p (sigmoid(z) - y)
__global__ void head_kernel(const float *h2, const float *w3, const float *b3, const float *y, const float *wt,
                            int32_t B, int32_t H, float *z, float *dz, float *loss) {
    const int p = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (p >= B) return;
    float s = 0.f;
    for (int i = lane; i < H; i += 32) s += h2[(size_t)p * H + i] * w3[i];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) {
        const float zz = s + b3[0];
        z[p] = zz;
        if (dz) {
            const float sg = 1.f / (1.f + __expf(-zz));
            const float w = wt ? wt[p] : 1.f;
            dz[p] = w * (sg - y[p]);
            // binary cross-entropy, numerically stable form
            const float l = fmaxf(zz, 0.f) - zz * y[p] + log1pf(__expf(-fabsf(zz)));
            atomicAdd(loss, w * l);
        }
    }
}

// x *= (h > 0): back through a ReLU whose output is h
__global__ void relu_back_kernel(float *x, const float *h, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(h[i] > 0.f)) x[i] = 0.f;
}

// Column sums of X[B][H], each row p optionally scaled by rowscale[p], in
// two deterministic stages: CTA (x, y) sums rows [y*rows_per, (y+1)*rows_per)
// of 32 columns (8 warps over interleaved rows, then the 8 warp sums in
// order) into part[y][H]; colsum_final_kernel adds the chunks in order.
constexpr int kColChunks = 32;
__global__ void __launch_bounds__(256) colsum_part_kernel(const float *X, const float *rowscale, int32_t B,
                                                          int32_t H, int32_t rows_per, float *part) {
    __shared__ float s[8][33];
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + lane;
    const int r0 = blockIdx.y * rows_per, r1 = min(B, r0 + rows_per);
    float sum = 0.f;
    if (col < H)
        for (int p = r0 + wy; p < r1; p += 8) sum += (rowscale ? rowscale[p] : 1.f) * X[(size_t)p * H + col];
    s[wy][lane] = sum;
    __syncthreads();
    if (wy == 0 && col < H) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += s[k][lane];
        part[(size_t)blockIdx.y * H + col] = t;
    }
}

__global__ void colsum_final_kernel(const float *part, int32_t R, int32_t H, float *out) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= H) return;
    float t = 0.f;
    for (int r = 0; r < R; ++r) t += part[(size_t)r * H + col];
    out[col] = t;
}

// dh2[p][i] = dz[p] * w3[i] where h2[p][i] > 0 (back through the head and
// the second ReLU), element-wise
__global__ void head_grad_kernel(const float *h2, const float *w3, const float *dz, int32_t B, int32_t H,
                                 float *dh2) {
    const size_t n = (size_t)B * H;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(i / H), c = (int)(i % H);
        dh2[i] = h2[i] > 0.f ? dz[p] * w3[c] : 0.f;
    }
}

// Adam (Kingma and Ba, 2015) on n parameters, gradient scaled by gscale
__global__ void adam_kernel(float *w, const float *gr, float *m, float *v, size_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2, float gscale) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float g = gr[i] * gscale;
        m[i] = b1 * m[i] + (1.f - b1) * g;
        v[i] = b2 * v[i] + (1.f - b2) * g * g;
        w[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
    }
}

// ------------------------------------------------------------ BF16 inference

// First layer on the tensor cores: H1[p][n] = relu(sum_f x_p[f] W1t[n][f] + b1[n])
// with x_p generated from the pair's truth vectors as 0/1 BF16 values (exact)
// and W1t = W1 transposed in BF16; mma.sync.m16n8k16 with FP32 accumulation.
// A CTA computes 64 pairs x 256 hidden units; warp w (of 8) owns hidden
// units [32w, 32w+32) for all 64 pairs (4 m-tiles x 4 n-tiles of 16x8).
constexpr int IBP = 64;           // pairs per CTA
constexpr int IBK = 32;           // features per k step (2 x k16)
constexpr int IH = 256;           // hidden width

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(256) infer_l1_bf16_kernel(const uint32_t *vec, int32_t vwords, const int32_t *pa,
                                                             const int32_t *pb, int32_t B,
                                                             const __nv_bfloat16 *w1t, const float *b1, float *h1) {
    __shared__ __nv_bfloat16 sx[IBP][IBK + 8];     // x tile: 64 pairs x 32 features
    __shared__ __nv_bfloat16 sw[IH][IBK + 8];      // W1t tile: 256 hidden x 32 features
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int p0 = blockIdx.x * IBP;
    const int F = vwords * 64;
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    const int half = vwords * 32;
    for (int f0 = 0; f0 < F; f0 += IBK) {
        // x tile: thread t < 64 builds pair t's 32 features from one word of each vector
        if (tid < IBP) {
            const int p = p0 + tid;
            uint32_t x = 0;
            if (p < B) {
                const int fb = f0 < half ? f0 : f0 - half;
                const uint32_t a = vec[(size_t)pa[p] * vwords + (fb >> 5)];
                const uint32_t b = vec[(size_t)pb[p] * vwords + (fb >> 5)];
                x = f0 < half ? (a ^ b) : (a & b);
            }
#pragma unroll
            for (int i = 0; i < IBK; ++i) sx[tid][i] = __float2bfloat16((float)((x >> i) & 1u));
        }
        // W1t tile: 256 rows x 32 bf16 = 16 KB, 4 x 16 bytes per thread
        for (int e = tid; e < IH * IBK / 8; e += 256) {
            const int r = e / (IBK / 8), c = (e % (IBK / 8)) * 8;
            *reinterpret_cast<uint4 *>(&sw[r][c]) = *reinterpret_cast<const uint4 *>(w1t + (size_t)r * F + f0 + c);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < IBK; kk += 16) {
            // fragments (PTX ISA m16n8k16 bf16 layouts): group g = lane/4, t = lane%4
            const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                uint32_t a[4];
                const int r0 = mt * 16 + gq;
                a[0] = *reinterpret_cast<const uint32_t *>(&sx[r0][kk + tq * 2]);
                a[1] = *reinterpret_cast<const uint32_t *>(&sx[r0 + 8][kk + tq * 2]);
                a[2] = *reinterpret_cast<const uint32_t *>(&sx[r0][kk + tq * 2 + 8]);
                a[3] = *reinterpret_cast<const uint32_t *>(&sx[r0 + 8][kk + tq * 2 + 8]);
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const int n0 = warp * 32 + nt * 8 + gq;
                    uint32_t b[2];
                    b[0] = *reinterpret_cast<const uint32_t *>(&sw[n0][kk + tq * 2]);
                    b[1] = *reinterpret_cast<const uint32_t *>(&sw[n0][kk + tq * 2 + 8]);
                    mma_bf16_16816(acc[mt][nt], a, b);
                }
            }
        }
        __syncthreads();
    }
    // C fragment: rows g and g+8, columns 2t, 2t+1
    const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int p = p0 + mt * 16 + gq + (r >= 2 ? 8 : 0);
                const int n = warp * 32 + nt * 8 + tq * 2 + (r & 1);
                if (p < B) {
                    const float v = acc[mt][nt][r] + b1[n];
                    h1[(size_t)p * IH + n] = v > 0.f ? v : 0.f;
                }
            }
}

__global__ void f32_to_bf16_t_kernel(const float *w, int32_t rows, int32_t cols, __nv_bfloat16 *wt) {
    // wt[c][r] = w[r][c]
    const size_t n = (size_t)rows * cols;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / cols, c = i % cols;
        wt[c * rows + r] = __float2bfloat16(w[i]);
    }
}

}  // namespace mkd

// ================================================================== host

using namespace mkd;

extern "C" int mk_fingerprint(const mk_program *d_progs, int32_t nprog, const mk_model *d_models,
                              const int32_t *h_group_n, int32_t ngroups, uint32_t *d_bits, int32_t *d_status,
                              void *stream) {
    if (nprog < 0 || ngroups < 0 || !h_group_n || !d_status) return MK_E_ARG;
    if (nprog == 0 || ngroups == 0) return MK_OK;
    if (!d_progs || !d_models || !d_bits) return MK_E_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int g = 0;
    while (g < ngroups) {
        const int n = h_group_n[g];
        if (n < 1 || n > MK_MAX_WORLDS_EXH) return MK_E_ARG;
        int e = g;
        while (e < ngroups && h_group_n[e] == n) ++e;
        dim3 grid((unsigned)((e - g + 127) / 128), (unsigned)((nprog + 63) / 64));
        switch (n) {
        case 1: fingerprint_kernel<1><<<grid, 128, 0, s>>>(d_progs, nprog, d_models, g, e - g, ngroups, d_bits, d_status); break;
        case 2: fingerprint_kernel<2><<<grid, 128, 0, s>>>(d_progs, nprog, d_models, g, e - g, ngroups, d_bits, d_status); break;
        case 3: fingerprint_kernel<3><<<grid, 128, 0, s>>>(d_progs, nprog, d_models, g, e - g, ngroups, d_bits, d_status); break;
        case 4: fingerprint_kernel<4><<<grid, 128, 0, s>>>(d_progs, nprog, d_models, g, e - g, ngroups, d_bits, d_status); break;
        case 5: fingerprint_kernel<5><<<grid, 128, 0, s>>>(d_progs, nprog, d_models, g, e - g, ngroups, d_bits, d_status); break;
        case 6: fingerprint_kernel<6><<<grid, 128, 0, s>>>(d_progs, nprog, d_models, g, e - g, ngroups, d_bits, d_status); break;
        }
        g = e;
    }
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

extern "C" size_t mk_knn_workspace_size(int32_t nvec) { return (size_t)nvec * (size_t)nvec * 2 + 256; }

extern "C" int mk_hamming_knn(const uint32_t *d_bits, int32_t nvec, int32_t words, int32_t k, int32_t *d_nbr,
                              uint16_t *d_dist, void *d_workspace, size_t ws_bytes, void *stream) {
    if (nvec < 2 || words < 1 || words > 1024 || k < 1 || !d_bits || !d_nbr || !d_dist) return MK_E_ARG;
    if (!d_workspace || ws_bytes < mk_knn_workspace_size(nvec)) return MK_E_WORKSPACE;
    const size_t sm = ((size_t)words * 32 + 1 + words) * 4;
    if (sm > 200 * 1024) return MK_E_ARG;
    ensure_dynamic_smem((const void *)knn_kernel, sm);
    knn_kernel<<<nvec, 512, sm, (cudaStream_t)stream>>>(d_bits, nvec, words, k, d_nbr, d_dist,
                                                        (uint16_t *)d_workspace);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

// ---- MLP: parameters in one FP32 buffer in the order W1 [F][H], b1 [H],
//      W2 [H][H], b2 [H], w3 [H], b3 [1]

namespace {

struct MlpView {
    int F, H;
    float *W1, *b1, *W2, *b2, *w3, *b3;
    size_t n;
};

MlpView mlp_view(float *base, int F, int H) {
    MlpView v;
    v.F = F;
    v.H = H;
    v.W1 = base;
    v.b1 = v.W1 + (size_t)F * H;
    v.W2 = v.b1 + H;
    v.b2 = v.W2 + (size_t)H * H;
    v.w3 = v.b2 + H;
    v.b3 = v.w3 + H;
    v.n = (size_t)F * H + H + (size_t)H * H + H + H + 1;
    return v;
}

template <int AM, int BM>
void gemm(const GemmArgs &g0, cudaStream_t s, float *part = nullptr, size_t part_floats = 0) {
    GemmArgs g = g0;
    const int ctas = ((g.N + GBN - 1) / GBN) * ((g.M + GBM - 1) / GBM);
    // a grid below two CTAs per SM splits K (chunks of at least 256, a
    // multiple of the k step) when the caller gave room for the partials
    int S = 1;
    if (part && ctas < kGemmFill && g.K >= 2 * kGemmMinChunk) {
        S = (kGemmFill + ctas - 1) / ctas;
        if (S > g.K / kGemmMinChunk) S = g.K / kGemmMinChunk;
        while (S > 1 && (size_t)S * g.M * g.N > part_floats) --S;
    }
    dim3 grid((unsigned)((g.N + GBN - 1) / GBN), (unsigned)((g.M + GBM - 1) / GBM), (unsigned)S);
    // the pair-feature operand has its own kernel (32-deep k steps)
    constexpr bool pair = (AM == A_PAIR || AM == A_PAIR_T) && BM == B_ROW;
    constexpr int step = pair ? PBK : GBK;
    auto launch = [&](const GemmArgs &a) {
        if constexpr (pair) {
            ensure_dynamic_smem((const void *)gemm_pair_kernel<AM == A_PAIR_T>, kPairSmem);
            gemm_pair_kernel<AM == A_PAIR_T><<<grid, 256, kPairSmem, s>>>(a);
        }
        else gemm_f32_kernel<AM, BM><<<grid, 256, 0, s>>>(a);
    };
    if (S == 1) {
        launch(g);
        return;
    }
    g.kchunk = ((g.K + S - 1) / S + step - 1) / step * step;
    g.part = part;
    launch(g);
    splitk_epilogue_kernel<<<1024, 256, 0, s>>>(part, S, g.M, g.N, g0.C, g0.ldc, g0.bias, g0.relu, g0.beta);
}

}  // namespace

extern "C" size_t mk_mlp_param_count(int32_t features, int32_t hidden) {
    return (size_t)features * hidden + hidden + (size_t)hidden * hidden + hidden + hidden + 1;
}

extern "C" size_t mk_mlp_workspace_size(int32_t batch, int32_t hidden) {
    return ((size_t)batch * hidden * 4 + (size_t)batch * 4) * sizeof(float) + 1024;
}

extern "C" int mk_mlp_forward(const float *d_params, int32_t features, int32_t hidden, const uint32_t *d_vec,
                              const int32_t *d_pa, const int32_t *d_pb, int32_t batch, float *d_logits,
                              void *d_workspace, size_t ws_bytes, void *stream) {
    if (features % 64 || hidden < 1 || batch < 0 || !d_params || !d_vec || !d_logits) return MK_E_ARG;
    if (batch == 0) return MK_OK;
    if (!d_workspace || ws_bytes < mk_mlp_workspace_size(batch, hidden)) return MK_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    MlpView v = mlp_view((float *)d_params, features, hidden);
    float *h1 = (float *)d_workspace, *h2 = h1 + (size_t)batch * hidden;
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.M = batch; g.N = hidden; g.K = features;
    g.vec = d_vec; g.pa = d_pa; g.pb = d_pb; g.vwords = features / 64;
    g.B = v.W1; g.ldb = hidden; g.C = h1; g.ldc = hidden; g.bias = v.b1; g.relu = 1;
    gemm<A_PAIR, B_ROW>(g, s);
    std::memset(&g, 0, sizeof(g));
    g.M = batch; g.N = hidden; g.K = hidden;
    g.A = h1; g.lda = hidden; g.B = v.W2; g.ldb = hidden; g.C = h2; g.ldc = hidden; g.bias = v.b2; g.relu = 1;
    gemm<A_ROW, B_ROW>(g, s);
    head_kernel<<<(batch + 7) / 8, 256, 0, s>>>(h2, v.w3, v.b3, nullptr, nullptr, batch, hidden, d_logits,
                                                 nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

namespace {

// Training workspace beyond the activations: split-K partials (up to
// kSplitCap copies of the largest GEMM output) and column-sum chunks.
constexpr size_t kSplitCap = 6;

size_t split_part_floats(int32_t batch, int32_t features, int32_t hidden) {
    const size_t a = (size_t)batch * hidden, b = (size_t)features * hidden;
    return kSplitCap * (a > b ? a : b);
}

size_t train_base_floats(int32_t batch, int32_t features, int32_t hidden) {
    return (size_t)batch * hidden * 4 + (size_t)batch * 4 + mk_mlp_param_count(features, hidden);
}

// Deterministic column sums of X[B][H] (rows optionally scaled) into out.
void colsum(const float *X, const float *rowscale, int32_t B, int32_t H, float *out, float *cpart, cudaStream_t s) {
    const int rows_per = (B + kColChunks - 1) / kColChunks;
    const int R = (B + rows_per - 1) / rows_per;
    colsum_part_kernel<<<dim3((unsigned)((H + 31) / 32), (unsigned)R), 256, 0, s>>>(X, rowscale, B, H, rows_per,
                                                                                      cpart);
    colsum_final_kernel<<<(H + 255) / 256, 256, 0, s>>>(cpart, R, H, out);
}

}  // namespace

extern "C" size_t mk_mlp_train_workspace_size(int32_t batch, int32_t features, int32_t hidden) {
    if (batch < 1 || features < 1 || hidden < 1) return 0;
    return (train_base_floats(batch, features, hidden) + split_part_floats(batch, features, hidden) +
            (size_t)kColChunks * (hidden > 1 ? hidden : 1) + 64) * sizeof(float) + 1024;
}

extern "C" int mk_mlp_gradient(const float *d_params, int32_t features, int32_t hidden, const uint32_t *d_vec,
                               const int32_t *d_pa, const int32_t *d_pb, const float *d_y, const float *d_w,
                               int32_t batch, float *d_grad, float *d_loss, void *d_workspace, size_t ws_bytes,
                               void *stream) {
    if (features % 64 || hidden < 1 || batch < 1 || !d_params || !d_vec || !d_y || !d_grad || !d_loss)
        return MK_E_ARG;
    if (!d_workspace || ws_bytes < mk_mlp_train_workspace_size(batch, features, hidden)) return MK_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const int H = hidden, F = features;
    MlpView v = mlp_view((float *)d_params, F, H);
    MlpView gv = mlp_view(d_grad, F, H);
    float *h1 = (float *)d_workspace, *h2 = h1 + (size_t)batch * H;
    float *dh1 = h2 + (size_t)batch * H, *dh2 = dh1 + (size_t)batch * H;
    float *z = dh2 + (size_t)batch * H, *dz = z + batch;
    float *part = (float *)d_workspace + ((train_base_floats(batch, F, H) + 63) & ~(size_t)63);
    const size_t part_floats = split_part_floats(batch, F, H);
    float *cpart = part + part_floats;
    cudaMemsetAsync(d_loss, 0, sizeof(float), s);
    GemmArgs g;
    // forward
    std::memset(&g, 0, sizeof(g));
    g.M = batch; g.N = H; g.K = F;
    g.vec = d_vec; g.pa = d_pa; g.pb = d_pb; g.vwords = F / 64;
    g.B = v.W1; g.ldb = H; g.C = h1; g.ldc = H; g.bias = v.b1; g.relu = 1;
    gemm<A_PAIR, B_ROW>(g, s, part, part_floats);
    std::memset(&g, 0, sizeof(g));
    g.M = batch; g.N = H; g.K = H;
    g.A = h1; g.lda = H; g.B = v.W2; g.ldb = H; g.C = h2; g.ldc = H; g.bias = v.b2; g.relu = 1;
    gemm<A_ROW, B_ROW>(g, s, part, part_floats);
    head_kernel<<<(batch + 7) / 8, 256, 0, s>>>(h2, v.w3, v.b3, d_y, d_w, batch, H, z, dz, d_loss);
    // backward: dh2, dw3 = sum_p dz[p] h2[p], db3 = sum_p dz[p]
    head_grad_kernel<<<1024, 256, 0, s>>>(h2, v.w3, dz, batch, H, dh2);
    colsum(h2, dz, batch, H, gv.w3, cpart, s);
    colsum(dz, nullptr, batch, 1, gv.b3, cpart, s);
    // dW2 = h1^T dh2 ; db2 = colsum dh2
    std::memset(&g, 0, sizeof(g));
    g.M = H; g.N = H; g.K = batch;
    g.A = h1; g.lda = H; g.B = dh2; g.ldb = H; g.C = gv.W2; g.ldc = H;
    gemm<A_COL, B_ROW>(g, s, part, part_floats);
    colsum(dh2, nullptr, batch, H, gv.b2, cpart, s);
    // dh1 = dh2 W2^T, then through the first ReLU
    std::memset(&g, 0, sizeof(g));
    g.M = batch; g.N = H; g.K = H;
    g.A = dh2; g.lda = H; g.B = v.W2; g.ldb = H; g.C = dh1; g.ldc = H;
    gemm<A_ROW, B_COL>(g, s, part, part_floats);
    relu_back_kernel<<<1024, 256, 0, s>>>(dh1, h1, (size_t)batch * H);
    // dW1 = X^T dh1 ; db1 = colsum dh1
    std::memset(&g, 0, sizeof(g));
    g.M = F; g.N = H; g.K = batch;
    g.vec = d_vec; g.pa = d_pa; g.pb = d_pb; g.vwords = F / 64;
    g.B = dh1; g.ldb = H; g.C = gv.W1; g.ldc = H;
    gemm<A_PAIR_T, B_ROW>(g, s, part, part_floats);
    colsum(dh1, nullptr, batch, H, gv.b1, cpart, s);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

extern "C" int mk_adam_step(float *d_params, const float *d_grad, float *d_m, float *d_v, size_t n, float lr,
                            float beta1, float beta2, float eps, int32_t step, float grad_scale, void *stream) {
    if (!d_params || !d_grad || !d_m || !d_v || step < 1) return MK_E_ARG;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<1024, 256, 0, (cudaStream_t)stream>>>(d_params, d_grad, d_m, d_v, n, lr, beta1, beta2, eps, c1, c2,
                                                        grad_scale);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

extern "C" size_t mk_mlp_infer_workspace_size(int32_t batch, int32_t features, int32_t hidden) {
    return ((size_t)batch * hidden * 2) * sizeof(float) + (size_t)features * hidden * 2 + 1024;
}

extern "C" int mk_mlp_infer_bf16(const float *d_params, int32_t features, int32_t hidden, const uint32_t *d_vec,
                                 const int32_t *d_pa, const int32_t *d_pb, int32_t batch, float *d_logits,
                                 void *d_workspace, size_t ws_bytes, void *stream) {
    if (hidden != IH || features % 64 || batch < 0 || !d_params || !d_vec || !d_logits) return MK_E_ARG;
    if (batch == 0) return MK_OK;
    if (!d_workspace || ws_bytes < mk_mlp_infer_workspace_size(batch, features, hidden)) return MK_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    MlpView v = mlp_view((float *)d_params, features, hidden);
    float *h1 = (float *)d_workspace, *h2 = h1 + (size_t)batch * hidden;
    __nv_bfloat16 *w1t = (__nv_bfloat16 *)(h2 + (size_t)batch * hidden);
    f32_to_bf16_t_kernel<<<1024, 256, 0, s>>>(v.W1, features, hidden, w1t);
    infer_l1_bf16_kernel<<<(batch + IBP - 1) / IBP, 256, 0, s>>>(d_vec, features / 64, d_pa, d_pb, batch, w1t,
                                                                  v.b1, h1);
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.M = batch; g.N = hidden; g.K = hidden;
    g.A = h1; g.lda = hidden; g.B = v.W2; g.ldb = hidden; g.C = h2; g.ldc = hidden; g.bias = v.b2; g.relu = 1;
    gemm<A_ROW, B_ROW>(g, s);
    head_kernel<<<(batch + 7) / 8, 256, 0, s>>>(h2, v.w3, v.b3, nullptr, nullptr, batch, hidden, d_logits, nullptr,
                                                 nullptr);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

// W1 (FP32, [features][hidden] in the parameter buffer) as BF16 W1^T.
extern "C" int mk_mlp_w1t_bf16(const float *d_params, int32_t features, int32_t hidden, void *d_w1t, void *stream) {
    if (features <= 0 || hidden <= 0 || !d_params || !d_w1t) return MK_E_ARG;
    MlpView v = mlp_view((float *)d_params, features, hidden);
    f32_to_bf16_t_kernel<<<1024, 256, 0, (cudaStream_t)stream>>>(v.W1, features, hidden, (__nv_bfloat16 *)d_w1t);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

// The first layer with warp-level mma.sync (the legacy tensor-core path),
// kept as the comparison for mk_mlp_layer1_tc.
extern "C" int mk_mlp_layer1_mma(const uint32_t *d_vec, int32_t features, const int32_t *d_pa, const int32_t *d_pb,
                                 int32_t batch, const void *d_w1t, const float *d_b1, float *d_h1, void *stream) {
    if (features <= 0 || features % 64 || batch < 0) return MK_E_ARG;
    if (batch == 0) return MK_OK;
    if (!d_vec || !d_pa || !d_pb || !d_w1t || !d_b1 || !d_h1) return MK_E_ARG;
    infer_l1_bf16_kernel<<<(batch + IBP - 1) / IBP, 256, 0, (cudaStream_t)stream>>>(
        d_vec, features / 64, d_pa, d_pb, batch, (const __nv_bfloat16 *)d_w1t, d_b1, d_h1);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

extern "C" int mk_mlp_infer_tc(const float *d_params, int32_t features, int32_t hidden, const uint32_t *d_vec,
                               const int32_t *d_pa, const int32_t *d_pb, int32_t batch, float *d_logits,
                               int32_t *d_status, void *d_workspace, size_t ws_bytes, void *stream) {
    if (hidden != IH || features % 128 || batch < 0 || !d_params || !d_vec || !d_logits || !d_status) return MK_E_ARG;
    if (batch == 0) return MK_OK;
    if (!d_workspace || ws_bytes < mk_mlp_infer_workspace_size(batch, features, hidden)) return MK_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    MlpView v = mlp_view((float *)d_params, features, hidden);
    float *h1 = (float *)d_workspace, *h2 = h1 + (size_t)batch * hidden;
    void *tiles = (void *)(h2 + (size_t)batch * hidden);            // features * hidden BF16, tiled
    int rc = mk_mlp_w1_tiles(d_params, features, hidden, tiles, stream);
    if (rc != MK_OK) return rc;
    rc = mk_mlp_layer1_tc_ws(d_vec, features, d_pa, d_pb, batch, tiles, v.b1, h1, d_status, stream);
    if (rc != MK_OK) return rc;
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.M = batch; g.N = hidden; g.K = hidden;
    g.A = h1; g.lda = hidden; g.B = v.W2; g.ldb = hidden; g.C = h2; g.ldc = hidden; g.bias = v.b2; g.relu = 1;
    gemm<A_ROW, B_ROW>(g, s);
    head_kernel<<<(batch + 7) / 8, 256, 0, s>>>(h2, v.w3, v.b3, nullptr, nullptr, batch, hidden, d_logits, nullptr,
                                                 nullptr);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}
