// Warm-start network on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// 16 inputs (9 features, zero padded) -> 4 hidden layers of 128 units (exact GELU) -> 16
// outputs (the first 3 used: n, u_y, T in normalised form).  Layer l: z_l = h_{l-1} W_l + b_l,
// W_l stored [inputs][outputs] in FP32 (master copy); BF16 operands, FP32 accumulation.
//
// Every GEMM is D[128 x N] (+)= A[128 x K] B[N x K]^T with A and B in shared memory in the
// K-major "core matrix" layout (8 rows x 16 bytes per 128-byte core matrix; neighbours along
// K 128 bytes apart, 8-row groups 16 K bytes apart), issued as tcgen05.mma kind::f16 (M = 128,
// K = 16 per instruction) by one thread, accumulated in tensor memory, completed through an
// mbarrier and read back with tcgen05.ld (thread t of the 128-thread block owns TMEM lane t).
//
// Forward: one block per 128-point tile, weights converted to BF16 in shared memory, the
// activation tile chained through one shared buffer.  Backward (training): per tile,
// dW_l = H_{l-1}^T dZ_l and dH_{l-1} = dZ_l W_l^T as tcgen05 GEMMs; each block writes its
// gradient to its own slot of a partial buffer, and the Adam kernel adds the slots in block
// order (deterministic) before the update.  This network has no counterpart in the paper.
#include "../../include/fdlb.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

namespace {

constexpr int NIN = 16, NH = 128, NOUT = 16, NUSED = 3;
// flat parameter offsets (W1, b1, ..., W5, b5)
constexpr int OW1 = 0, OB1 = OW1 + NIN * NH;
constexpr int OW2 = OB1 + NH, OB2 = OW2 + NH * NH;
constexpr int OW3 = OB2 + NH, OB3 = OW3 + NH * NH;
constexpr int OW4 = OB3 + NH, OB4 = OW4 + NH * NH;
constexpr int OW5 = OB4 + NH, OB5 = OW5 + NH * NOUT;
constexpr int NPARAM = OB5 + NOUT;                 // 53776
constexpr int TILE = 128;
constexpr int WAIT_LIMIT = 4000000;                // bounded mbarrier wait

__host__ __device__ constexpr int woff(int l) { return l == 1 ? OW1 : l == 2 ? OW2 : l == 3 ? OW3 : l == 4 ? OW4 : OW5; }
__host__ __device__ constexpr int boff(int l) { return l == 1 ? OB1 : l == 2 ? OB2 : l == 3 ? OB3 : l == 4 ? OB4 : OB5; }

// byte offset of element (r, k) of an operand with K columns in the core-matrix layout
__device__ __forceinline__ int cm(int r, int k, int K) { return (r >> 3) * (16 * K) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, int K) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((128 >> 4) & 0x3FFF) << 16;          // leading byte offset: K-neighbour core matrices
    d |= (uint64_t)(((16 * K) >> 4) & 0x3FFF) << 32;     // stride byte offset: 8-row groups
    d |= (uint64_t)1 << 46;                               // descriptor version
    return d;                                             // no swizzle
}

__device__ __forceinline__ uint32_t idesc(int N) {
    // FP32 accumulate, BF16 A and B, both K-major, N >> 3, M = 128 >> 4
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TILE >> 4) << 24);
}

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// D(tmem) (+)= A(smem, 128 x K) B(smem, N x K)^T, issued by the calling thread.
__device__ __forceinline__ void mma(uint32_t tmem, const unsigned char* A, const unsigned char* B, int K, int N, bool acc) {
    const uint32_t a0 = saddr(A), b0 = saddr(B), id = idesc(N);
    for (int s = 0; s < K / 16; ++s) {
        const uint64_t ad = sdesc(a0 + s * 256, K), bd = sdesc(b0 + s * 256, K);
        const uint32_t en = (acc || s > 0) ? 1u : 0u;
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                     :: "r"(tmem), "l"(ad), "l"(bd), "r"(id), "r"(en) : "memory");
    }
}

__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(saddr(bar)) : "memory");
}

// Wait for phase `parity` of the mbarrier, at most WAIT_LIMIT polls; false on timeout.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < WAIT_LIMIT && !done; ++it)
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(saddr(bar)), "r"(parity) : "memory");
    return done != 0;
}

__device__ __forceinline__ void sync_for_mma() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, int cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(saddr(slot)), "r"(cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t tmem, int cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(cols) : "memory");
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ void put_bf16(unsigned char* base, int off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}

// ------------------------------------------------------------------------------ packed weights
// The BF16 core-matrix images of the weights that the forward and backward kernels use as
// GEMM operands, written once per call from the FP32 master copy (k_mlp_pack) and copied into
// each block's shared memory with bulk asynchronous copies.
constexpr int PK_FWD = 106496;                 // W1t, W2t..W4t, W5t (the forward's first bytes)
constexpr int PK_BWD = 102400;                 // W2n..W4n, W5n (the backward's first bytes)
constexpr int PK_BYTES = PK_FWD + PK_BWD;

__device__ __forceinline__ void bulk_copy(unsigned char* dst, const unsigned char* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(saddr(dst)), "l"(src), "r"(bytes), "r"(saddr(bar)) : "memory");
}

// bytes (a multiple of 4096, 16-byte aligned at both ends) into shared memory by the block's
// threads, 4 KB per copy; false when the copies did not complete within the wait limit
__device__ bool load_packed(unsigned char* dst, const unsigned char* src, int bytes, uint64_t* cbar) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(cbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(saddr(cbar)), "r"((uint32_t)bytes) : "memory");
    }
    __syncthreads();
    for (int c = tid; c < bytes / 4096; c += blockDim.x) bulk_copy(dst + c * 4096, src + c * 4096, 4096, cbar);
    return __syncthreads_and(wait_bar(cbar, 0) ? 1 : 0) != 0;
}

__global__ void k_mlp_pack(const float* __restrict__ prm, unsigned char* __restrict__ pk) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned char* fw = pk;
    unsigned char* bw = pk + PK_FWD;
    // forward operands B = W_l^T (rows: outputs, K = inputs); backward B = W_l (rows: inputs,
    // K = outputs) for l >= 2; byte offsets as in the kernels' shared-memory layouts
    if (e < OB1) {
        const int k = e / NH, n = e % NH;
        put_bf16(fw, cm(n, k, NIN), prm[e]);
    } else {
        for (int l = 2; l <= 4; ++l) {
            const int q = e - woff(l);
            if (q >= 0 && q < NH * NH) {
                const int a = q / NH, b = q % NH;
                put_bf16(fw + 4096 + (l - 2) * 32768, cm(b, a, NH), prm[e]);
                put_bf16(bw + (l - 2) * 32768, cm(a, b, NH), prm[e]);
            }
        }
        const int q = e - OW5;
        if (q >= 0 && q < NH * NOUT) {
            const int a = q / NOUT, b = q % NOUT;
            put_bf16(fw + 4096 + 3 * 32768, cm(b, a, NH), prm[e]);
            put_bf16(bw + 3 * 32768, cm(a, b, NOUT), prm[e]);
        }
    }
}

// ------------------------------------------------------------------------------ forward
// Shared bytes: W1t 4096 | W2t..W4t 3 x 32768 | W5t 4096 | A 32768 | bias 2112
constexpr int F_W1 = 0, F_W2 = 4096, F_W3 = F_W2 + 32768, F_W4 = F_W3 + 32768, F_W5 = F_W4 + 32768;
constexpr int F_A = F_W5 + 4096, F_BIAS = F_A + 32768, F_BYTES = F_BIAS + 4 * 4 * NH + 4 * NOUT;

__global__ void __launch_bounds__(TILE) k_mlp_fwd(const float* __restrict__ prm, const unsigned char* __restrict__ pk,
                                                  const float* __restrict__ X, int P, float* __restrict__ pred,
                                                  float* __restrict__ Zs, int* err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar, cbar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x;
    const int p = blockIdx.x * TILE + tid;
    const bool valid = p < P;
    if (tid < 32) tmem_alloc(&tslot, NH);
    // weights as B operands (N = outputs x K = inputs): the packed BF16 image, biases
    static_assert(F_A == PK_FWD, "packed forward image = the weight region of shared memory");
    bool ok = load_packed(sm, pk, PK_FWD, &cbar);
    float* bias = reinterpret_cast<float*>(sm + F_BIAS);
    for (int e = tid; e < 4 * NH + NOUT; e += TILE) bias[e] = e < 4 * NH ? prm[boff(e / NH + 1) + e % NH] : prm[OB5 + e - 4 * NH];
    // input tile (K = 16)
    for (int k = 0; k < NIN; ++k) put_bf16(sm + F_A, cm(tid, k, NIN), valid ? X[(size_t)p * NIN + k] : 0.0f);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    sync_for_mma();
    const uint32_t tmem = tslot;
    const uint32_t lane_addr = tmem + ((uint32_t)((tid >> 5) * 32) << 16);
    for (int l = 1; l <= 5 && ok; ++l) {
        const int K = l == 1 ? NIN : NH, N = l == 5 ? NOUT : NH;
        const unsigned char* W = sm + (l == 1 ? F_W1 : l == 2 ? F_W2 : l == 3 ? F_W3 : l == 4 ? F_W4 : F_W5);
        if (tid == 0) {
            mma(tmem, sm + F_A, W, K, N, false);
            commit(&bar);
        }
        ok = __syncthreads_and(wait_bar(&bar, (uint32_t)((l - 1) & 1)) ? 1 : 0) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) break;                      // uniform across the block
        const float* bl = bias + (l - 1) * NH;
        for (int c0 = 0; c0 < N; c0 += 32) {
            float v[32];
            tmem_ld32(lane_addr + c0, v);    // 32 columns (all inside the 128 allocated)
            const int cn = N - c0 < 32 ? N - c0 : 32;
            for (int j = 0; j < cn; ++j) {
                const int c = c0 + j;
                const float z = v[j] + bl[c];
                if (l < 5) {
                    if (Zs && valid) Zs[(size_t)p * 4 * NH + (l - 1) * NH + c] = z;
                    put_bf16(sm + F_A, cm(tid, c, NH), gelu(z));
                } else if (c < NUSED && valid) {
                    pred[(size_t)p * NUSED + c] = z;
                }
            }
        }
        sync_for_mma();
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid < 32) tmem_free(tmem, NH);
}

// ------------------------------------------------------------------------------ backward
// Shared bytes: W2n..W4n 3 x 32768 (natural: N = inputs x K = outputs) | W5n 4096 (N = 128 x K = 16)
//               | OpA 32768 | OpB 32768 | OpC 32768
constexpr int B_W2 = 0, B_W3 = 32768, B_W4 = 65536, B_W5 = 98304, B_A = B_W5 + 4096, B_B = B_A + 32768, B_C = B_B + 32768;
constexpr int B_BYTES = B_C + 32768;

__global__ void __launch_bounds__(TILE) k_mlp_bwd(const unsigned char* __restrict__ pk, const float* __restrict__ X,
                                                  const float* __restrict__ Y, int P, const float* __restrict__ pred,
                                                  const float* __restrict__ Zs, float* __restrict__ gpart,
                                                  float* __restrict__ lpart, int* err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar, cbar;
    __shared__ uint32_t tslot;
    __shared__ float red[TILE / 32];
    const int tid = threadIdx.x;
    const int p = blockIdx.x * TILE + tid;
    const bool valid = p < P;
    float* g = gpart + (size_t)blockIdx.x * NPARAM;
    if (tid < 32) tmem_alloc(&tslot, 2 * NH);
    // weights as B operands of the dH GEMMs (N = inputs x K = outputs): the packed BF16 image
    static_assert(B_A == PK_BWD, "packed backward image = the weight region of shared memory");
    bool ok = load_packed(sm, pk + PK_FWD, PK_BWD, &cbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // dZ_5 = dL/dpred on the used outputs; loss partial
    float d[NH];
    float sq = 0.0f;
#pragma unroll
    for (int j = 0; j < NH; ++j) d[j] = 0.0f;
    if (valid)
        for (int j = 0; j < NUSED; ++j) {
            const float df = pred[(size_t)p * NUSED + j] - Y[(size_t)p * NUSED + j];
            sq += df * df;
            d[j] = 2.0f * df / (float)(NUSED * P);
        }
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((tid & 31) == 0) red[tid >> 5] = sq;
    sync_for_mma();
    if (tid == 0) lpart[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
    const uint32_t tmem = tslot;
    const uint32_t lane_addr = tmem + ((uint32_t)((tid >> 5) * 32) << 16);
    uint32_t phase = 0;
    for (int l = 5; l >= 1 && ok; --l) {
        const int N = l == 5 ? NOUT : NH;          // outputs of layer l
        // operands: dW GEMM  A = H_{l-1}^T (rows: inputs), B = dZ^T (rows: outputs), K = points;
        //           layer 1: A = dZ_1^T (rows: outputs), B = X^T (rows: inputs).
        //           dH GEMM  A = dZ (rows: points, K = outputs), B = W_l natural (rows: inputs).
        if (l >= 2) {
            for (int c = 0; c < NH; ++c) {
                const float z = valid ? Zs[(size_t)p * 4 * NH + (l - 2) * NH + c] : 0.0f;
                put_bf16(sm + B_A, cm(c, tid, TILE), valid ? gelu(z) : 0.0f);
            }
            for (int j = 0; j < N; ++j) {
                put_bf16(sm + B_B, cm(j, tid, TILE), d[j]);
                put_bf16(sm + B_C, cm(tid, j, N), d[j]);
            }
        } else {
            for (int j = 0; j < NH; ++j) put_bf16(sm + B_A, cm(j, tid, TILE), d[j]);
            for (int k = 0; k < NIN; ++k) put_bf16(sm + B_B, cm(k, tid, TILE), valid ? X[(size_t)p * NIN + k] : 0.0f);
        }
        sync_for_mma();
        if (tid == 0) {
            mma(tmem, sm + B_A, sm + B_B, TILE, l >= 2 ? N : NIN, false);
            if (l >= 2) mma(tmem + NH, sm + B_C, sm + (l == 2 ? B_W2 : l == 3 ? B_W3 : l == 4 ? B_W4 : B_W5), N, NH, false);
            commit(&bar);
        }
        ok = __syncthreads_and(wait_bar(&bar, phase) ? 1 : 0) != 0;
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) break;                      // uniform across the block
        // weight gradient: row tid of the dW accumulator
        const int NW = l >= 2 ? N : NIN;
        for (int c0 = 0; c0 < NW; c0 += 32) {
            float v[32];
            tmem_ld32(lane_addr + c0, v);        // 32 columns inside the dW accumulator's 128
            const int cn = NW - c0 < 32 ? NW - c0 : 32;
            for (int j = 0; j < cn; ++j) {
                const int c = c0 + j;
                if (l >= 2) g[woff(l) + tid * N + c] = v[j];          // dW_l[in = tid][out = c]
                else g[OW1 + c * NH + tid] = v[j];                    // dW_1[in = c][out = tid]
            }
        }
        // bias gradient: column sums of dZ_l over the tile's points
        {
            const unsigned char* src = sm + (l >= 2 ? B_B : B_A);
            if (tid < N) {
                float s = 0.0f;
                for (int q = 0; q < TILE; ++q) s += __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(src + cm(tid, q, TILE)));
                g[boff(l) + tid] = s;
            }
        }
        if (l >= 2) {
            // dH_{l-1} (row = point), then dZ_{l-1} = dH * GELU'(Z_{l-1})
            for (int c0 = 0; c0 < NH; c0 += 32) {
                float v[32];
                tmem_ld32(lane_addr + NH + c0, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float z = valid ? Zs[(size_t)p * 4 * NH + (l - 2) * NH + c0 + j] : 0.0f;
                    d[c0 + j] = valid ? v[j] * gelu_grad(z) : 0.0f;
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid < 32) tmem_free(tmem, 2 * NH);
}

// ------------------------------------------------------------------------------ Adam
__global__ void k_mlp_adam(float* prm, float* m, float* v, const float* gpart, int nblk, float lr, float b1t, float b2t,
                           float* gout) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= NPARAM) return;
    float gsum = 0.0f;
    for (int b = 0; b < nblk; ++b) gsum += gpart[(size_t)b * NPARAM + q];
    if (gout) gout[q] = gsum;
    if (lr == 0.0f) return;
    const float mq = 0.9f * m[q] + 0.1f * gsum;
    const float vq = 0.999f * v[q] + 0.001f * gsum * gsum;
    m[q] = mq;
    v[q] = vq;
    prm[q] -= lr * (mq / (1.0f - b1t)) / (sqrtf(vq / (1.0f - b2t)) + 1e-8f);
}

// Glorot-uniform weights from a counter-based hash (splitmix64 of seed and index), zero biases;
// output columns beyond the 3 used are zero.
__global__ void k_mlp_init(float* prm, float* m, float* v, unsigned long long seed) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= NPARAM) return;
    m[q] = 0.0f;
    v[q] = 0.0f;
    int l = 5;
    for (int j = 1; j <= 5; ++j)
        if (q < boff(j) + (j == 5 ? NOUT : NH)) { l = j; break; }
    if (q >= boff(l)) { prm[q] = 0.0f; return; }
    const int fin = l == 1 ? NIN : NH, fout = l == 5 ? NOUT : NH;
    if (l == 5 && (q - OW5) % NOUT >= NUSED) { prm[q] = 0.0f; return; }
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(q + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float u = (float)((z >> 40) * (1.0 / 16777216.0)) * 2.0f - 1.0f;
    prm[q] = u * sqrtf(6.0f / (float)(fin + fout));
}

}  // namespace

// ------------------------------------------------------------------------------ C ABI
struct fdlb_mlp {
    float* prm = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* gpart = nullptr;
    float* lpart = nullptr;
    float* Zs = nullptr;
    float* pred = nullptr;
    int* err = nullptr;
    unsigned char* pk = nullptr;      // packed BF16 weight images (k_mlp_pack)
    int max_points = 0;
    long long t = 0;
    cudaStream_t stream = nullptr;
    std::string msg;
};

static thread_local std::string g_mlp_err;

static size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

static size_t mlp_layout(int max_points, size_t* off) {
    const size_t nblk = (size_t)(max_points + TILE - 1) / TILE;
    size_t o = 0;
    off[0] = o; o += al256(sizeof(float) * NPARAM);               // parameters
    off[1] = o; o += al256(sizeof(float) * NPARAM);               // Adam m
    off[2] = o; o += al256(sizeof(float) * NPARAM);               // Adam v
    off[3] = o; o += al256(sizeof(float) * NPARAM * nblk);        // per-block gradients
    off[4] = o; o += al256(sizeof(float) * nblk);                 // per-block loss
    off[5] = o; o += al256(sizeof(float) * 4 * NH * (size_t)max_points);   // pre-activations
    off[6] = o; o += al256(sizeof(float) * NUSED * (size_t)max_points);    // predictions
    off[7] = o; o += al256(sizeof(int));
    off[8] = o; o += al256(PK_BYTES);                            // packed BF16 weight images
    return o;
}

static int mlp_fail(fdlb_mlp* h, int code, const std::string& s) {
    if (h) h->msg = s;
    g_mlp_err = s;
    return code;
}

static int mlp_cuda(fdlb_mlp* h, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return FDLB_OK;
    return mlp_fail(h, FDLB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

extern "C" int32_t fdlb_mlp_param_count(void) { return NPARAM; }

extern "C" size_t fdlb_mlp_workspace_bytes(int32_t max_points) {
    if (max_points < 1) return 0;
    size_t off[9];
    return mlp_layout(max_points, off);
}

extern "C" const char* fdlb_mlp_last_error(const fdlb_mlp* h) { return h ? h->msg.c_str() : g_mlp_err.c_str(); }

extern "C" int fdlb_mlp_create(fdlb_mlp** out, void* dev_ws, size_t bytes, int32_t max_points, uint64_t seed, void* stream) {
    if (!out || !dev_ws || max_points < 1) return mlp_fail(nullptr, FDLB_EINVAL, "fdlb_mlp_create: bad arguments");
    size_t off[9];
    const size_t need = mlp_layout(max_points, off);
    if (bytes < need || (reinterpret_cast<uintptr_t>(dev_ws) & 255))
        return mlp_fail(nullptr, FDLB_ENOMEM, "fdlb_mlp_create: workspace smaller than fdlb_mlp_workspace_bytes or misaligned");
    fdlb_mlp* h = new fdlb_mlp();
    char* b = static_cast<char*>(dev_ws);
    h->prm = reinterpret_cast<float*>(b + off[0]);
    h->m = reinterpret_cast<float*>(b + off[1]);
    h->v = reinterpret_cast<float*>(b + off[2]);
    h->gpart = reinterpret_cast<float*>(b + off[3]);
    h->lpart = reinterpret_cast<float*>(b + off[4]);
    h->Zs = reinterpret_cast<float*>(b + off[5]);
    h->pred = reinterpret_cast<float*>(b + off[6]);
    h->err = reinterpret_cast<int*>(b + off[7]);
    h->pk = reinterpret_cast<unsigned char*>(b + off[8]);
    h->max_points = max_points;
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    int rc = mlp_cuda(h, cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, F_BYTES), "attributes");
    if (!rc) rc = mlp_cuda(h, cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, B_BYTES), "attributes");
    if (!rc) {
        k_mlp_init<<<(NPARAM + 255) / 256, 256, 0, h->stream>>>(h->prm, h->m, h->v, (unsigned long long)seed);
        rc = mlp_cuda(h, cudaGetLastError(), "init kernel");
    }
    if (!rc) rc = mlp_cuda(h, cudaMemsetAsync(h->err, 0, sizeof(int), h->stream), "clear");
    if (!rc) rc = mlp_cuda(h, cudaStreamSynchronize(h->stream), "synchronize");
    if (rc) { g_mlp_err = h->msg; delete h; return rc; }
    *out = h;
    return FDLB_OK;
}

extern "C" void fdlb_mlp_destroy(fdlb_mlp* h) { delete h; }

extern "C" int fdlb_mlp_get_params(fdlb_mlp* h, float* host) {
    if (!h || !host) return mlp_fail(h, FDLB_EINVAL, "fdlb_mlp_get_params: bad arguments");
    int rc = mlp_cuda(h, cudaMemcpyAsync(host, h->prm, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, h->stream), "copy");
    if (!rc) rc = mlp_cuda(h, cudaStreamSynchronize(h->stream), "synchronize");
    return rc;
}

extern "C" int fdlb_mlp_set_params(fdlb_mlp* h, const float* host) {
    if (!h || !host) return mlp_fail(h, FDLB_EINVAL, "fdlb_mlp_set_params: bad arguments");
    int rc = mlp_cuda(h, cudaMemcpyAsync(h->prm, host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, h->stream), "copy");
    if (!rc) rc = mlp_cuda(h, cudaMemsetAsync(h->m, 0, sizeof(float) * NPARAM, h->stream), "clear");
    if (!rc) rc = mlp_cuda(h, cudaMemsetAsync(h->v, 0, sizeof(float) * NPARAM, h->stream), "clear");
    if (!rc) rc = mlp_cuda(h, cudaStreamSynchronize(h->stream), "synchronize");
    h->t = 0;
    return rc;
}

static int check_err(fdlb_mlp* h) {
    int e = 0;
    int rc = mlp_cuda(h, cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "copy");
    if (!rc) rc = mlp_cuda(h, cudaStreamSynchronize(h->stream), "synchronize");
    if (!rc && e) rc = mlp_fail(h, FDLB_ETIMEOUT, "tensor-core completion wait timed out");
    return rc;
}

extern "C" int fdlb_mlp_predict(fdlb_mlp* h, const float* dev_x, int32_t points, float* dev_y) {
    if (!h || !dev_x || !dev_y || points < 1) return mlp_fail(h, FDLB_EINVAL, "fdlb_mlp_predict: bad arguments");
    const int nblk = (points + TILE - 1) / TILE;
    k_mlp_pack<<<(NPARAM + 255) / 256, 256, 0, h->stream>>>(h->prm, h->pk);
    k_mlp_fwd<<<nblk, TILE, F_BYTES, h->stream>>>(h->prm, h->pk, dev_x, points, dev_y, nullptr, h->err);
    int rc = mlp_cuda(h, cudaGetLastError(), "forward kernel");
    if (!rc) rc = check_err(h);
    return rc;
}

extern "C" int fdlb_mlp_train_step(fdlb_mlp* h, const float* dev_x, const float* dev_y, int32_t points, float lr,
                                   float* dev_grad, double* host_loss) {
    if (!h || !dev_x || !dev_y || points < 1 || points > h->max_points || !(lr >= 0.0f))
        return mlp_fail(h, FDLB_EINVAL, "fdlb_mlp_train_step: bad arguments (points must be <= max_points)");
    const int nblk = (points + TILE - 1) / TILE;
    k_mlp_pack<<<(NPARAM + 255) / 256, 256, 0, h->stream>>>(h->prm, h->pk);
    k_mlp_fwd<<<nblk, TILE, F_BYTES, h->stream>>>(h->prm, h->pk, dev_x, points, h->pred, h->Zs, h->err);
    k_mlp_bwd<<<nblk, TILE, B_BYTES, h->stream>>>(h->pk, dev_x, dev_y, points, h->pred, h->Zs, h->gpart, h->lpart, h->err);
    if (lr > 0.0f) h->t += 1;
    const float b1t = lr > 0.0f ? (float)std::pow(0.9, (double)h->t) : 0.0f;
    const float b2t = lr > 0.0f ? (float)std::pow(0.999, (double)h->t) : 0.0f;
    k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, h->stream>>>(h->prm, h->m, h->v, h->gpart, nblk, lr, b1t, b2t, dev_grad);
    int rc = mlp_cuda(h, cudaGetLastError(), "training kernels");
    if (!rc && host_loss) {
        std::vector<float> lp(nblk);
        rc = mlp_cuda(h, cudaMemcpyAsync(lp.data(), h->lpart, sizeof(float) * nblk, cudaMemcpyDeviceToHost, h->stream), "copy");
        if (!rc) rc = mlp_cuda(h, cudaStreamSynchronize(h->stream), "synchronize");
        double s = 0.0;
        for (float x : lp) s += x;
        if (!rc) *host_loss = s / (NUSED * (double)points);
    }
    if (!rc) rc = check_err(h);
    return rc;
}
