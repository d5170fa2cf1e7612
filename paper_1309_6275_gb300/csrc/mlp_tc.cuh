// mlp_tc.cuh -- the proposal network's forward pass on the 5th-generation
// tensor cores (included by mlp.cu).  Layers 2 and 3 are dense contractions
// (128 hits x 128 x 128 and 128 x 128 x 64 per tile): one thread issues
// tcgen05.mma (kind::f16, BF16 operands from shared memory, float32
// accumulators in tensor memory), the four warps read the accumulators back
// with tcgen05.ld (warp w holds rows 32w..32w+31, thread = hit) for the
// bias, ReLU, BF16 rounding and softmax epilogues.  Layer 1 (6 inputs) runs
// on the CUDA cores.  Operands sit in shared memory in the no-swizzle
// K-major core-matrix layout: 8 rows x 16 bytes per 128-byte core matrix,
// core matrices adjacent along K 128 bytes apart (leading byte offset),
// along M/N 2048 bytes apart (stride byte offset).  Every wait on the MMA
// completion barrier is bounded; on expiry the kernel counts a timeout,
// frees its tensor memory and returns.

constexpr int kTcM = 128;                         // hits per tile (MMA M)
constexpr uint32_t kTcCols = 256;                 // tensor-memory columns per CTA
constexpr uint32_t kLBO = 128, kSBO = 2048;       // core-matrix strides (K = 128)
constexpr size_t kTcSmem = (size_t)kH * kH * 2 + (size_t)kOut * kH * 2 + (size_t)kTcM * kH * 2 +
                           (size_t)kIn * kH * 2 + (size_t)(2 * kH + kOut + kOut) * 4 + 64;
constexpr long long kTcSpin = 1ll << 22;          // bounded barrier wait (~0.5 s)

__device__ unsigned int g_mlp_timeouts;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row, k) of a K = 128 operand in the core layout.
__device__ __forceinline__ uint32_t core_off(int row, int k)
{
    return (uint32_t)((row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start >> 4, LBO >> 4, SBO >> 4, version 1,
// no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((kLBO >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((kSBO >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: float32 accumulator, BF16 A and B, both
// K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 lanes x 32 columns of 32 bits: thread i of the warp gets row lane0 + i.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
                 "tcgen05.wait::ld.sync.aligned;\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr)
                 : "memory");
}

// Wait for phase `phase` of the barrier; false when the bound expires.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase)
{
    for (long long i = 0; i < kTcSpin; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Store 8 BF16 values (columns c .. c + 7 of `row`) into a core-layout tile.
__device__ __forceinline__ void st_core8(unsigned char *tile, int row, int c, const float v[8])
{
    __align__(16) __nv_bfloat16 b[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) b[u] = __float2bfloat16_rn(v[u]);
    *reinterpret_cast<uint4 *>(tile + core_off(row, c)) = *reinterpret_cast<const uint4 *>(b);
}

__global__ void __launch_bounds__(kTcM)
k_mlp_fwd_tc(const __nv_bfloat16 *__restrict__ w, const float *__restrict__ x,
             const float *__restrict__ y, const float *__restrict__ z,
             const uint8_t *__restrict__ layer, int n, FwdOut out)
{
    // no-swizzle core-matrix operands need 16-byte alignment only
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *sB2 = smem;                                   // W2^T: N 128 x K 128
    unsigned char *sB3 = sB2 + kH * kH * 2;                      // W3^T: N 64 x K 128
    unsigned char *sA = sB3 + kOut * kH * 2;                     // activations: 128 x 128
    __nv_bfloat16 *sW1 = reinterpret_cast<__nv_bfloat16 *>(sA + kTcM * kH * 2);
    float *sb1 = reinterpret_cast<float *>(sW1 + kIn * kH);
    float *sb2 = sb1 + kH, *sb3 = sb2 + kH, *smass = sb3 + kOut;
    __shared__ __align__(8) unsigned long long s_mbar;
    __shared__ uint32_t s_tmem;
    __shared__ int sev;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (out.d_n) n = *out.d_n;

    for (int t = tid; t < kH * kH; t += kTcM) {                  // B2(n = o, k = i) = W2[i][o]
        const int i = t / kH, o = t % kH;
        *reinterpret_cast<__nv_bfloat16 *>(sB2 + core_off(o, i)) = w[oW2 + t];
    }
    for (int t = tid; t < kH * kOut; t += kTcM) {                // B3(n = c, k = i) = W3[i][c]
        const int i = t / kOut, c = t % kOut;
        *reinterpret_cast<__nv_bfloat16 *>(sB3 + core_off(c, i)) = w[oW3 + t];
    }
    for (int t = tid; t < kIn * kH; t += kTcM) sW1[t] = w[oW1 + t];
    for (int t = tid; t < kH; t += kTcM) {
        sb1[t] = __bfloat162float(w[ob1 + t]);
        sb2[t] = __bfloat162float(w[ob2 + t]);
    }
    for (int t = tid; t < kOut; t += kTcM) sb3[t] = __bfloat162float(w[ob3 + t]);
    const uint32_t mbar = smem_u32(&s_mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&s_tmem)), "r"(kTcCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // weights -> tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t d2 = tmem, d3 = tmem + kH;                    // columns [0,128), [128,192)
    const uint32_t row_base = (uint32_t)(warp * 32) << 16;       // this warp's TMEM lanes
    const uint32_t aA = smem_u32(sA), aB2 = smem_u32(sB2), aB3 = smem_u32(sB3);
    uint32_t phase = 0;
    bool failed = false;

    for (int base = blockIdx.x * kTcM; base < n; base += gridDim.x * kTcM) {
        const int h = base + tid;
        const bool act = h < n;
        // ---- features and layer 1 (CUDA cores) into the A tile
        float f[kIn];
        hit_features(act ? x[h] : 0.f, act ? y[h] : 0.f, act ? z[h] : 0.f, act ? layer[h] : 0, f);
        if (act && out.feat) {
            __align__(16) __nv_bfloat16 fb[8];
#pragma unroll
            for (int i = 0; i < kIn; ++i) fb[i] = __float2bfloat16_rn(f[i]);
            fb[6] = fb[7] = __float2bfloat16_rn(0.f);
            *reinterpret_cast<uint4 *>(out.feat + (size_t)h * 8) = *reinterpret_cast<uint4 *>(fb);
        }
        for (int o0 = 0; o0 < kH; o0 += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                float a = sb1[o0 + u];
#pragma unroll
                for (int i = 0; i < kIn; ++i) a = fmaf(f[i], __bfloat162float(sW1[i * kH + o0 + u]), a);
                v[u] = fmaxf(a, 0.f);
            }
            st_core8(sA, tid, o0, v);
            if (act && out.h1) {
                __align__(16) __nv_bfloat16 b[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) b[u] = __float2bfloat16_rn(v[u]);
                *reinterpret_cast<uint4 *>(out.h1 + (size_t)h * kH + o0) = *reinterpret_cast<uint4 *>(b);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // A tile -> tensor cores
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- layer 2: D2 = A x B2 (M 128, N 128, K 128 in 8 steps of 16)
        if (tid == 0) {
#pragma unroll
            for (int kk = 0; kk < kH / 16; ++kk)
                tc_mma(d2, smem_desc(aA + kk * 2 * kLBO), smem_desc(aB2 + kk * 2 * kLBO),
                       mma_idesc(kTcM, kH), kk > 0);
            tc_commit(mbar);
        }
        if (!__syncthreads_and(mbar_wait(mbar, phase))) {   // the same decision everywhere
            failed = true;
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        // ---- epilogue 2: bias, ReLU, BF16 -> A tile (layer 3's operand)
        for (int c0 = 0; c0 < kH; c0 += 32) {
            uint32_t r[32];
            tc_ld32(d2 + row_base + c0, r);
#pragma unroll
            for (int q = 0; q < 32; q += 8) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    v[u] = fmaxf(__uint_as_float(r[q + u]) + sb2[c0 + q + u], 0.f);
                st_core8(sA, tid, c0 + q, v);
                if (act && out.h2) {
                    __align__(16) __nv_bfloat16 b[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) b[u] = __float2bfloat16_rn(v[u]);
                    *reinterpret_cast<uint4 *>(out.h2 + (size_t)h * kH + c0 + q) =
                        *reinterpret_cast<uint4 *>(b);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- layer 3: D3 = A x B3 (M 128, N 64, K 128)
        if (tid == 0) {
#pragma unroll
            for (int kk = 0; kk < kH / 16; ++kk)
                tc_mma(d3, smem_desc(aA + kk * 2 * kLBO), smem_desc(aB3 + kk * 2 * kLBO),
                       mma_idesc(kTcM, kOut), kk > 0);
            tc_commit(mbar);
        }
        if (!__syncthreads_and(mbar_wait(mbar, phase))) {   // the same decision everywhere
            failed = true;
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        // ---- epilogue 3: logits, softmax (thread = hit)
        float lg[kOut];
#pragma unroll
        for (int c0 = 0; c0 < kOut; c0 += 32) {
            uint32_t r[32];
            tc_ld32(d3 + row_base + c0, r);
#pragma unroll
            for (int q = 0; q < 32; ++q) lg[c0 + q] = __uint_as_float(r[q]) + sb3[c0 + q];
        }
        float mx = lg[0];
#pragma unroll
        for (int c = 1; c < kOut; ++c) mx = fmaxf(mx, lg[c]);
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < kOut; ++c) {
            lg[c] = __expf(lg[c] - mx);
            s += lg[c];
        }
        const float is = __frcp_rn(s);
#pragma unroll
        for (int c = 0; c < kOut; ++c) lg[c] *= is;
        if (act && out.hmask) {
            // top-k regions: k passes of a first-maximum scan (ties go to the
            // smaller region), then the fallback on their summed probability
            unsigned long long sel = ~0ull;
            if (out.topk < kOut) {
                sel = 0ull;
                float sum = 0.f;
                for (int t = 0; t < out.topk; ++t) {
                    float best = -1.f;
                    int bi = 0;
#pragma unroll
                    for (int c = 0; c < kOut; ++c) {
                        if (!((sel >> c) & 1ull) && lg[c] > best) {
                            best = lg[c];
                            bi = c;
                        }
                    }
                    sel |= 1ull << bi;
                    sum += best;
                }
                if (sum < out.pmin) sel = ~0ull;
            }
            out.hmask[h] = sel;
        }
        if (act && out.prob) {
            float4 *pp = reinterpret_cast<float4 *>(out.prob + (size_t)h * kOut);
#pragma unroll
            for (int c4 = 0; c4 < kOut / 4; ++c4)
                pp[c4] = make_float4(lg[4 * c4], lg[4 * c4 + 1], lg[4 * c4 + 2], lg[4 * c4 + 3]);
        }
        if (out.mass) {
            if (tid == 0) sev = event_of_hit(out.off, out.n_ev, base);
            for (int c = tid; c < kOut; c += kTcM) smass[c] = 0.f;
            __syncthreads();
            const int e = act ? event_of_hit(out.off, out.n_ev, h) : -1;
            if (__all_sync(0xffffffffu, !act || e == sev)) {
                // the warp's hits are all in event sev: reduce-scatter the 64
                // sums over the warp (halves exchanged with lane ^ 16, 8, 4,
                // 2, 1; the lane with that bit set keeps the upper half),
                // after which lane l holds the sums of regions 2l and 2l + 1
                const int lane = tid & 31;
#pragma unroll
                for (int c = 0; c < kOut; ++c) lg[c] = act ? lg[c] : 0.f;
#pragma unroll
                for (int st = 0; st < 5; ++st) {
                    const int hs = 32 >> st, po = 16 >> st;
                    const bool up = (lane & po) != 0;
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        if (i < hs) {
                            const float send = up ? lg[i] : lg[i + hs];
                            const float keep = up ? lg[i + hs] : lg[i];
                            lg[i] = keep + __shfl_xor_sync(0xffffffffu, send, po);
                        }
                    }
                }
                const int c0 = 2 * lane;
                atomicAdd(&smass[c0], lg[0]);
                atomicAdd(&smass[c0 + 1], lg[1]);
            } else if (act) {
                if (e == sev) {
#pragma unroll
                    for (int c = 0; c < kOut; ++c) atomicAdd(&smass[c], lg[c]);
                } else {
#pragma unroll
                    for (int c = 0; c < kOut; ++c) atomicAdd(&out.mass[(size_t)e * kOut + c], lg[c]);
                }
            }
            __syncthreads();
            for (int c = tid; c < kOut; c += kTcM) atomicAdd(&out.mass[(size_t)sev * kOut + c], smass[c]);
        }
        tc_fence_before();
        __syncthreads();      // all reads of D2/D3 and of the A tile done before reuse
        tc_fence_after();
    }
    if (failed) {
        // count it, give the outstanding MMAs one more bounded wait, then free
        if (tid == 0) atomicAdd(&g_mlp_timeouts, 1u);
        mbar_wait(mbar, phase);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTcCols) : "memory");
}

// ---------------------------------------------------------------------------
// Training contractions on the tensor cores.
//
// Backward through the activations (k_mlp_bwd_tc), per tile of 128 hits:
//   dL  = (p - onehot) / nl                      (CUDA cores, thread = hit)
//   dH2 = (dL W3^T) o [h2 > 0]    M 128, N 128, K 64  (tcgen05)
//   dH1 = (dH2 W2^T) o [h1 > 0]   M 128, N 128, K 128 (tcgen05)
// with W3 stored [hidden][class] and W2 [in][out], so both B operands are
// the stored rows (n = the hidden unit, k contiguous).  dL and dH2 enter the
// tensor cores rounded to BF16; the accumulators and the stored gradients
// are float32.
//
// Weight gradients (k_wgrad_tc): C[m][n] = sum_h A[h][m] B[h][n] for one
// split of the hits, M = 128, N = 128 or 64, K = 128 hits per step: A^T and
// B^T are staged K-major (eight hits per 16-byte core-matrix row) and the
// split's sum accumulates in tensor memory.  B (a float32 gradient) enters
// rounded to BF16; the bias sum over the same hits is float32 in hit order.
// Splits are reduced in a fixed order (k_wgrad_reduce), so a training step is
// reproducible bit for bit.

constexpr uint32_t kSBO64 = 1024;                 // 8-row group stride for K = 64
constexpr size_t kBwdTcSmem = (size_t)kH * kOut * 2 + (size_t)kH * kH * 2 +
                              (size_t)kTcM * kOut * 2 + (size_t)kTcM * kH * 2;
constexpr size_t kWgTcSmem = (size_t)kTcM * kTcM * 2 + (size_t)kH * kTcM * 2;
constexpr uint32_t kWgTcCols = 128;

// Byte offset of element (row, k) of a K = 64 operand in the core layout.
__device__ __forceinline__ uint32_t core_off64(int row, int k)
{
    return (uint32_t)((row >> 3) * kSBO64 + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc_sbo(uint32_t addr, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((kLBO >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// One CTA's tensor-memory columns and completion barrier (warp 0 allocates).
__device__ __forceinline__ uint32_t tc_setup(uint32_t mbar, uint32_t *s_tmem, uint32_t cols)
{
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(s_tmem)), "r"(cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *s_tmem;
}

// After a bounded wait failed: count it, one more bounded wait for the
// outstanding MMAs; then (every path) free the tensor memory.
__device__ __forceinline__ void tc_teardown(bool failed, uint32_t mbar, uint32_t phase,
                                            uint32_t tmem, uint32_t cols)
{
    if (failed) {
        if (threadIdx.x == 0) atomicAdd(&g_mlp_timeouts, 1u);
        mbar_wait(mbar, phase);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(cols) : "memory");
}

// The operand writes above are visible to the tensor cores, and every
// thread reaches the MMA issue point.
__device__ __forceinline__ void tc_publish()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__global__ void __launch_bounds__(kTcM)
k_mlp_bwd_tc(const __nv_bfloat16 *__restrict__ w, const float *__restrict__ prob,
             const int *__restrict__ labels, const __nv_bfloat16 *__restrict__ h1,
             const __nv_bfloat16 *__restrict__ h2, int n, const int *__restrict__ d_nlab,
             float *__restrict__ dL, float *__restrict__ dH2, float *__restrict__ dH1)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *sB3 = smem;                          // W3: N 128 (hidden) x K 64 (class)
    unsigned char *sB2 = sB3 + kH * kOut * 2;           // W2: N 128 (in) x K 128 (out)
    unsigned char *sA1 = sB2 + kH * kH * 2;             // dL: 128 hits x K 64
    unsigned char *sA2 = sA1 + kTcM * kOut * 2;         // dH2: 128 hits x K 128
    __shared__ __align__(8) unsigned long long s_mbar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int t = tid; t < kH * kOut; t += kTcM)         // B3(n = o, k = c) = W3[o][c]
        *reinterpret_cast<__nv_bfloat16 *>(sB3 + core_off64(t / kOut, t % kOut)) = w[oW3 + t];
    for (int t = tid; t < kH * kH; t += kTcM)           // B2(n = i, k = o) = W2[i][o]
        *reinterpret_cast<__nv_bfloat16 *>(sB2 + core_off(t / kH, t % kH)) = w[oW2 + t];
    const uint32_t mbar = smem_u32(&s_mbar);
    const uint32_t tmem = tc_setup(mbar, &s_tmem, kTcCols);
    const uint32_t d1 = tmem, d2 = tmem + kH;
    const uint32_t row_base = (uint32_t)(warp * 32) << 16;
    const uint32_t aA1 = smem_u32(sA1), aA2 = smem_u32(sA2), aB3 = smem_u32(sB3),
                   aB2 = smem_u32(sB2);
    const float inv_nl = 1.0f / (float)max(*d_nlab, 1);
    uint32_t phase = 0;
    bool failed = false;
    for (int base = blockIdx.x * kTcM; base < n; base += gridDim.x * kTcM) {
        const int h = base + tid;
        const bool act = h < n;
        const int lab = act ? labels[h] : -1;
        // ---- dL (thread = hit): global float32, BF16 into the A tile
        for (int c0 = 0; c0 < kOut; c0 += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float pv = act ? prob[(size_t)h * kOut + c0 + u] : 0.f;
                v[u] = lab >= 0 ? (pv - (c0 + u == lab ? 1.f : 0.f)) * inv_nl : 0.f;
            }
            if (act) {
                float4 *dp = reinterpret_cast<float4 *>(dL + (size_t)h * kOut + c0);
                dp[0] = make_float4(v[0], v[1], v[2], v[3]);
                dp[1] = make_float4(v[4], v[5], v[6], v[7]);
            }
            __align__(16) __nv_bfloat16 b[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) b[u] = __float2bfloat16_rn(v[u]);
            *reinterpret_cast<uint4 *>(sA1 + core_off64(tid, c0)) = *reinterpret_cast<uint4 *>(b);
        }
        tc_publish();
        // ---- D1 = dL x W3^T (M 128, N 128, K 64 in 4 steps of 16)
        if (tid == 0) {
#pragma unroll
            for (int kk = 0; kk < kOut / 16; ++kk)
                tc_mma(d1, smem_desc_sbo(aA1 + kk * 2 * kLBO, kSBO64),
                       smem_desc_sbo(aB3 + kk * 2 * kLBO, kSBO64), mma_idesc(kTcM, kH), kk > 0);
            tc_commit(mbar);
        }
        if (!__syncthreads_and(mbar_wait(mbar, phase))) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        // ---- dH2 = D1 o [h2 > 0]: global float32, BF16 into the second A tile
        for (int c0 = 0; c0 < kH; c0 += 32) {
            uint32_t r[32];
            tc_ld32(d1 + row_base + c0, r);
#pragma unroll
            for (int q = 0; q < 32; q += 8) {
                __align__(16) __nv_bfloat16 hv[8];
                *reinterpret_cast<uint4 *>(hv) =
                    act ? *reinterpret_cast<const uint4 *>(h2 + (size_t)h * kH + c0 + q)
                        : make_uint4(0, 0, 0, 0);
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    v[u] = __bfloat162float(hv[u]) > 0.f ? __uint_as_float(r[q + u]) : 0.f;
                if (act) {
                    float4 *dp = reinterpret_cast<float4 *>(dH2 + (size_t)h * kH + c0 + q);
                    dp[0] = make_float4(v[0], v[1], v[2], v[3]);
                    dp[1] = make_float4(v[4], v[5], v[6], v[7]);
                }
                st_core8(sA2, tid, c0 + q, v);
            }
        }
        tc_publish();
        // ---- D2 = dH2 x W2^T (M 128, N 128, K 128)
        if (tid == 0) {
#pragma unroll
            for (int kk = 0; kk < kH / 16; ++kk)
                tc_mma(d2, smem_desc(aA2 + kk * 2 * kLBO), smem_desc(aB2 + kk * 2 * kLBO),
                       mma_idesc(kTcM, kH), kk > 0);
            tc_commit(mbar);
        }
        if (!__syncthreads_and(mbar_wait(mbar, phase))) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        // ---- dH1 = D2 o [h1 > 0]
        for (int c0 = 0; c0 < kH; c0 += 32) {
            uint32_t r[32];
            tc_ld32(d2 + row_base + c0, r);
#pragma unroll
            for (int q = 0; q < 32; q += 8) {
                if (!act) continue;
                __align__(16) __nv_bfloat16 hv[8];
                *reinterpret_cast<uint4 *>(hv) =
                    *reinterpret_cast<const uint4 *>(h1 + (size_t)h * kH + c0 + q);
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    v[u] = __bfloat162float(hv[u]) > 0.f ? __uint_as_float(r[q + u]) : 0.f;
                float4 *dp = reinterpret_cast<float4 *>(dH1 + (size_t)h * kH + c0 + q);
                dp[0] = make_float4(v[0], v[1], v[2], v[3]);
                dp[1] = make_float4(v[4], v[5], v[6], v[7]);
            }
        }
        tc_fence_before();
        __syncthreads();      // D1, D2 and both A tiles are free again
        tc_fence_after();
    }
    tc_teardown(failed, mbar, phase, tmem, kTcCols);
}

// Split blockIdx.x of C[128][N] = sum_h A[h][m] B[h][n] (A BF16, row stride
// lda; B float32, row stride ldb) and of bias[n] = sum_h B[h][n], over the
// split's hits; stored at C + split pstride and bias + split pstride.
__global__ void __launch_bounds__(kTcM)
k_wgrad_tc(const __nv_bfloat16 *__restrict__ A, int lda, const float *__restrict__ B, int ldb,
           int n, int N, float *__restrict__ C, float *__restrict__ bias, size_t pstride)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *sA = smem;                           // A^T: M 128 x K 128 hits
    unsigned char *sB = smem + kTcM * kTcM * 2;         // B^T: N x K 128 hits
    __shared__ __align__(8) unsigned long long s_mbar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5;
    C += (size_t)blockIdx.x * pstride;
    bias += (size_t)blockIdx.x * pstride;
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int h0 = blockIdx.x * per, h1 = min(n, h0 + per);
    const uint32_t mbar = smem_u32(&s_mbar);
    const uint32_t tmem = tc_setup(mbar, &s_tmem, kWgTcCols);
    const uint32_t aA = smem_u32(sA), aB = smem_u32(sB);
    uint32_t phase = 0;
    bool failed = false, any = false;
    float bacc = 0.f;
    for (int hb = h0; hb < h1; hb += kTcM) {
        // ---- stage: thread = row m of A^T (and n of B^T), eight hits per store
        for (int g = 0; g < kTcM / 8; ++g) {
            __align__(16) __nv_bfloat16 av[8], bv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int hh = hb + 8 * g + u;
                const bool in = hh < h1;
                av[u] = in ? A[(size_t)hh * lda + tid] : __float2bfloat16_rn(0.f);
                float b = 0.f;
                if (tid < N && in) b = B[(size_t)hh * ldb + tid];
                bacc += b;
                bv[u] = __float2bfloat16_rn(b);
            }
            *reinterpret_cast<uint4 *>(sA + core_off(tid, 8 * g)) = *reinterpret_cast<uint4 *>(av);
            if (tid < N)
                *reinterpret_cast<uint4 *>(sB + core_off(tid, 8 * g)) =
                    *reinterpret_cast<uint4 *>(bv);
        }
        tc_publish();
        if (tid == 0) {
#pragma unroll
            for (int kk = 0; kk < kTcM / 16; ++kk)
                tc_mma(tmem, smem_desc(aA + kk * 2 * kLBO), smem_desc(aB + kk * 2 * kLBO),
                       mma_idesc(kTcM, N), (any || kk > 0) ? 1u : 0u);
            tc_commit(mbar);
        }
        any = true;
        if (!__syncthreads_and(mbar_wait(mbar, phase))) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc_fence_after();   // the tiles may be overwritten: the MMAs are done
    }
    if (!failed) {
        // thread = row m: the split's sums (zero when it had no hits)
        for (int c0 = 0; c0 < N; c0 += 32) {
            uint32_t r[32];
            if (any) tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, r);
#pragma unroll
            for (int q = 0; q < 32; ++q)
                C[(size_t)tid * N + c0 + q] = any ? __uint_as_float(r[q]) : 0.f;
        }
        if (tid < N) bias[tid] = bacc;
    }
    tc_teardown(failed, mbar, phase, tmem, kWgTcCols);
}
