// tn_tc.cu -- tensor-core node kernel (tcgen05 + TMEM) for large nodes.
//
// A large tree node (Sec. 2 of arXiv 2002.01935: the inner product of two
// tensors over their shared labels) is a batched GEMM C[b] = A[b] B[b]
// whose operands are read through the same bit-scatter offsets as the
// CUDA-core tile kernel.  Here the product runs on the 5th-generation
// tensor cores:
//   * four producer warps gather A and B tiles from global memory, split
//     each value into hi + lo parts (TF32 or BF16, round to nearest), and
//     store them into shared memory in the K-major, 128-byte-swizzled
//     layout that tcgen05.mma reads;
//   * one MMA warp issues tcgen05.mma (kind::tf32 or kind::f16 with BF16)
//     into an FP32 accumulator tile in tensor memory: hi*hi + hi*lo +
//     lo*hi for the split modes, a single product otherwise;
//   * the producer warps then read the accumulator with tcgen05.ld, apply
//     the power-of-two renormalisation and write C.
// Complex nodes use one real GEMM with K doubled (4M): A is read as
// interleaved (re, im) pairs along K, and B is expanded in shared memory
// into rows (Re B, -Im B) and (Im B, Re B), so the accumulator holds
// interleaved (re, im) outputs.
// Every mbarrier wait is bounded; on timeout the kernel records TN_ETIMEOUT
// in the control block, waits (bounded) for its MMAs, frees its tensor
// memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tn.h"
#include "tn_internal.h"

namespace tn {

namespace {

constexpr int kBM = 128;          // accumulator rows (TMEM lanes)
constexpr int kBN = 128;          // accumulator columns (real)
constexpr int kRowBytes = 128;    // one swizzle row per stage and operand
constexpr int kTileBytes = kBM * kRowBytes;  // 16 KB per operand part
constexpr int kProducers = 512;   // 16 warps
constexpr int kThreads = kProducers + 32;
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false after ~kWaitCycles (the caller aborts).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    long long t0 = clock64();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 255) == 255) {
            if (*abort_flag) return false;
            if (clock64() - t0 > kWaitCycles) return false;
        }
    }
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)2 << 61;              // SWIZZLE_128B
    return d;
}

// Instruction descriptor: FP32 accumulator, A/B format, K-major both,
// N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t instr_desc(uint32_t ab_format, int M, int N) {
    return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate) {
    if constexpr (BF16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ int64_t scatter(uint64_t x, const uint8_t* sh, int nbits) {
    int64_t o = 0;
    for (int i = 0; i < nbits; ++i)
        if (((x >> i) & 1ull) && sh[i] != kNoBit) o += (int64_t)1 << sh[i];
    return o;
}

__device__ __forceinline__ int64_t slice_offset(const SliceDigits& d, int64_t slice) {
    int64_t off = 0;
    for (int i = 0; i < d.n; ++i) off += ((slice / d.div[i]) % d.dim[i]) * d.stride[i];
    return off;
}

__device__ __forceinline__ int exp_of(const unsigned* slot) {
    if (slot == nullptr) return 0;
    float m = __uint_as_float(*slot);
    if (!(m > 0.f)) return 0;
    int e;
    frexpf(m, &e);
    return e;
}

// Round to TF32 (10 explicit mantissa bits), nearest with ties away.
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// 16-byte chunk position of (row, chunk) in a 128B-swizzled K-major tile.
__device__ __forceinline__ uint32_t swz(int row, int chunk) {
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

// hi/lo parts of four real values into 16 bytes each (TF32: 4 floats).
template <bool BF16>
struct Pack;
template <>
struct Pack<false> {
    // 4 values -> one 16B chunk
    static __device__ __forceinline__ void split4(const float* x, uint4& hi, uint4& lo, bool split) {
        float h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            h[i] = to_tf32(x[i]);
            l[i] = split ? to_tf32(x[i] - h[i]) : 0.f;
        }
        hi = make_uint4(__float_as_uint(h[0]), __float_as_uint(h[1]), __float_as_uint(h[2]),
                        __float_as_uint(h[3]));
        lo = make_uint4(__float_as_uint(l[0]), __float_as_uint(l[1]), __float_as_uint(l[2]),
                        __float_as_uint(l[3]));
    }
};
template <>
struct Pack<true> {
    // 8 values -> one 16B chunk
    static __device__ __forceinline__ void split8(const float* x, uint4& hi, uint4& lo) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * i]);
            __nv_bfloat16 h1 = __float2bfloat16_rn(x[2 * i + 1]);
            __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * i] - __bfloat162float(h0));
            __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * i + 1] - __bfloat162float(h1));
            h[i] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            l[i] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
        hi = make_uint4(h[0], h[1], h[2], h[3]);
        lo = make_uint4(l[0], l[1], l[2], l[3]);
    }
};

}  // namespace

// PREC: 0 = TF32 single product, 1 = TF32 hi+lo (3 products),
//       2 = BF16 hi+lo (3 products).
template <bool CPLX, int PREC, int STAGES>
__global__ void __launch_bounds__(kThreads, 1) k_tc(const __grid_constant__ TileArgs a) {
    constexpr bool BF16 = PREC == 2;
    constexpr bool SPLIT = PREC != 0;
    constexpr int PARTS = SPLIT ? 2 : 1;                 // hi (+ lo) per operand
    constexpr int STAGE_BYTES = 2 * PARTS * kTileBytes;  // A and B
    // real K per stage: a 128-byte row holds 32 TF32 or 64 BF16 values
    constexpr int KR = BF16 ? 64 : 32;
    constexpr int KC = CPLX ? KR / 2 : KR;               // source (complex) K per stage
    constexpr int NC = CPLX ? kBN / 2 : kBN;             // source N per tile
    constexpr int MMA_K = BF16 ? 16 : 8;                 // real K per instruction
    constexpr int KSTEPS = KR / MMA_K;                   // instructions per part pair
    constexpr uint32_t FMT = BF16 ? 1u : 2u;

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ int64_t rowA[kBM], colB[NC], kA[KC], kB[KC];

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int64_t M = 1ll << a.nm, N = 1ll << a.nn, K = 1ll << a.nk;
    const int64_t tiles_n = (N + NC - 1) / NC;
    const int64_t m0 = ((int64_t)blockIdx.x / tiles_n) * kBM;
    const int64_t n0 = ((int64_t)blockIdx.x % tiles_n) * NC;
    const int64_t b = blockIdx.z % a.nbatch;
    const int inst = (int)(blockIdx.z / a.nbatch);
    const int nkb = (int)((K + KC - 1) / KC);
    // this instance's operands, result, scale slots and slice (an idle
    // instance leaves before touching barriers or tensor memory)
    const InstanceInfo& in = a.in;
    const int64_t slice = a.ctl->slice + (int64_t)inst * in.slice_step;
    if (slice >= a.ctl->slice_end) return;
    constexpr int ESZ = CPLX ? 8 : 4;
    const void* Ainst = (const char*)a.A + (int64_t)inst * in.a_is * ESZ;
    const void* Binst = (const char*)a.B + (int64_t)inst * in.b_is * ESZ;
    void* Cinst = (char*)a.C + (int64_t)inst * in.c_is * ESZ;
    ScaleIO sio = a.sc;
    if (sio.max_a) sio.max_a += (int64_t)inst * in.sa_is;
    if (sio.exp_a) sio.exp_a += (int64_t)inst * in.sa_is;
    if (sio.max_b) sio.max_b += (int64_t)inst * in.sb_is;
    if (sio.exp_b) sio.exp_b += (int64_t)inst * in.sb_is;
    sio.max_c += (int64_t)inst * in.sc_is;
    sio.exp_c += (int64_t)inst * in.sc_is;

    // renormalisation of the operands (exact powers of two)
    const int eA = exp_of(sio.max_a), eB = exp_of(sio.max_b);
    const int cA = max(-120, min(120, eA)), cB = max(-120, min(120, eB));
    const float fa = ldexpf(1.f, -cA), fb = ldexpf(1.f, -cB);
    const int resid = (eA - cA) + (eB - cB);
    if (blockIdx.x == 0 && b == 0 && tid == 0 && sio.exp_c)
        *sio.exp_c = (sio.exp_a ? *sio.exp_a : 0) + (sio.exp_b ? *sio.exp_b : 0) + eA + eB;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], kProducers);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
    }
    for (int i = tid; i < kBM; i += kThreads) rowA[i] = scatter(i, a.a_m, a.nm);
    for (int j = tid; j < NC; j += kThreads) colB[j] = scatter(j, a.b_n, a.nn);
    for (int t = tid; t < KC; t += kThreads) {
        kA[t] = scatter(t, a.a_k, a.nk);
        kB[t] = scatter(t, a.b_k, a.nk);
    }
    constexpr int kMmaWarp = kProducers / 32;
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(kBN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == kMmaWarp) {
        // ---------------- MMA issuer ----------------
        if ((tid & 31) == 0) {
            const uint32_t idesc = instr_desc(FMT, kBM, kBN);
            bool ok = true;
            for (int kb = 0; kb < nkb && ok; ++kb) {
                const int s = kb % STAGES;
                if (!mbar_wait(&full_bar[s], (uint32_t)((kb / STAGES) & 1), &abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
                const uint32_t a_hi = base, b_hi = base + PARTS * kTileBytes;
                const uint32_t a_lo = base + kTileBytes, b_lo = b_hi + kTileBytes;
#pragma unroll
                for (int k = 0; k < KSTEPS; ++k) {
                    const uint32_t off = k * MMA_K * (BF16 ? 2 : 4);
                    const uint32_t acc0 = (kb > 0 || k > 0) ? 1u : 0u;
                    mma<BF16>(tmem, smem_desc(a_hi + off), smem_desc(b_hi + off), idesc, acc0);
                    if constexpr (SPLIT) {
                        mma<BF16>(tmem, smem_desc(a_hi + off), smem_desc(b_lo + off), idesc, 1u);
                        mma<BF16>(tmem, smem_desc(a_lo + off), smem_desc(b_hi + off), idesc, 1u);
                    }
                }
                mma_commit(&empty_bar[s]);
            }
            if (!ok) {
                abort_flag = 1;
                atomicExch(const_cast<int32_t*>(&a.ctl->status), (int32_t)TN_ETIMEOUT);
            }
            mma_commit(&done_bar);
        }
        __syncwarp();
    } else {
        // ---------------- producers ----------------
        const float* Af = reinterpret_cast<const float*>(Ainst);
        const float* Bf = reinterpret_cast<const float*>(Binst);
        const int64_t baseA = slice_offset(a.sla, slice) + scatter(b, a.a_b, a.nb) + scatter(m0, a.a_m, a.nm);
        const int64_t baseB = slice_offset(a.slb, slice) + scatter(b, a.b_b, a.nb) + scatter(n0, a.b_n, a.nn);
        const int mlim = (int)min(M - m0, (int64_t)kBM);
        const int nlim = (int)min(N - n0, (int64_t)NC);
        constexpr int VPC = BF16 ? 8 : 4;      // real values per 16B chunk
        constexpr int CPC = CPLX ? VPC / 2 : VPC;  // source values per chunk (A)
        constexpr int A_ITEMS = kBM * 8 / kProducers;             // 16B chunks per thread
        constexpr int BROWS = CPLX ? kBN / 2 : kBN;
        constexpr int B_ITEMS = BROWS * 8 / kProducers;
        constexpr int BPC = CPLX ? CPC : VPC;                    // source values per B item
        constexpr int BV = CPLX ? CPC * 2 : VPC;                 // floats loaded per B item
        struct Regs {
            float a[A_ITEMS][VPC];
            float b[B_ITEMS][BV];
        };
        // per-thread operand offsets: an item's rows and K positions are the
        // same in every k-block (only the k-block base moves)
        const int kmax = (int)min(K, (int64_t)KC);
        int32_t oa[A_ITEMS][CPC], ob[B_ITEMS][BPC];
        uint32_t va = 0, vb = 0;  // validity bits
#pragma unroll
        for (int i = 0; i < A_ITEMS; ++i) {
            const int it = tid + i * kProducers;
            const int r = a.a_mfast ? it % kBM : it / 8;
            const int c = a.a_mfast ? it / kBM : it % 8;
#pragma unroll
            for (int v = 0; v < CPC; ++v) {
                const int kk = c * CPC + v;
                const bool in = r < mlim && kk < kmax;
                oa[i][v] = in ? (int32_t)(rowA[r] + kA[kk]) : 0;
                va |= (in ? 1u : 0u) << (i * CPC + v);
            }
        }
#pragma unroll
        for (int i = 0; i < B_ITEMS; ++i) {
            const int it = tid + i * kProducers;
            const int j = a.b_nfast ? it % BROWS : it / 8;
            const int c = a.b_nfast ? it / BROWS : it % 8;
#pragma unroll
            for (int v = 0; v < BPC; ++v) {
                const int kk = c * BPC + v;
                const bool in = j < nlim && kk < kmax;
                ob[i][v] = in ? (int32_t)(colB[j] + kB[kk]) : 0;
                vb |= (in ? 1u : 0u) << (i * BPC + v);
            }
        }
        // issue every gather of k-block kb into registers
        auto gather = [&](int kb, Regs& R) {
            const int64_t k0 = (int64_t)kb * KC;
            const float* pa = Af + (baseA + scatter(k0, a.a_k, a.nk)) * (CPLX ? 2 : 1);
            const float* pb = Bf + (baseB + scatter(k0, a.b_k, a.nk)) * (CPLX ? 2 : 1);
#pragma unroll
            for (int i = 0; i < A_ITEMS; ++i)
#pragma unroll
                for (int v = 0; v < CPC; ++v) {
                    const bool in = (va >> (i * CPC + v)) & 1u;
                    if constexpr (CPLX) {
                        const float2 z = in ? reinterpret_cast<const float2*>(pa)[oa[i][v]] : make_float2(0.f, 0.f);
                        R.a[i][2 * v] = z.x;
                        R.a[i][2 * v + 1] = a.conj_a ? -z.y : z.y;
                    } else {
                        R.a[i][v] = in ? pa[oa[i][v]] : 0.f;
                    }
                }
#pragma unroll
            for (int i = 0; i < B_ITEMS; ++i)
#pragma unroll
                for (int v = 0; v < BPC; ++v) {
                    const bool in = (vb >> (i * BPC + v)) & 1u;
                    if constexpr (CPLX) {
                        const float2 z = in ? reinterpret_cast<const float2*>(pb)[ob[i][v]] : make_float2(0.f, 0.f);
                        R.b[i][2 * v] = z.x;
                        R.b[i][2 * v + 1] = a.conj_b ? -z.y : z.y;
                    } else {
                        R.b[i][v] = in ? pb[ob[i][v]] : 0.f;
                    }
                }
        };
        // scale, split and store k-block kb into its stage, then signal it
        auto deposit = [&](int kb, const Regs& R) -> bool {
            const int s = kb % STAGES;
            if (kb >= STAGES && !mbar_wait(&empty_bar[s], (uint32_t)(((kb / STAGES) + 1) & 1), &abort_flag))
                return false;
            uint8_t* st = smem + s * STAGE_BYTES;
#pragma unroll
            for (int i = 0; i < A_ITEMS; ++i) {
                const int it = tid + i * kProducers;
                const int r = a.a_mfast ? it % kBM : it / 8;
                const int c = a.a_mfast ? it / kBM : it % 8;
                float x[VPC];
#pragma unroll
                for (int v = 0; v < VPC; ++v) x[v] = R.a[i][v] * fa;
                uint4 hi, lo;
                if constexpr (BF16) Pack<true>::split8(x, hi, lo);
                else Pack<false>::split4(x, hi, lo, SPLIT);
                *reinterpret_cast<uint4*>(st + swz(r, c)) = hi;
                if constexpr (SPLIT) *reinterpret_cast<uint4*>(st + kTileBytes + swz(r, c)) = lo;
            }
            uint8_t* sb = st + PARTS * kTileBytes;
#pragma unroll
            for (int i = 0; i < B_ITEMS; ++i) {
                const int it = tid + i * kProducers;
                const int j = a.b_nfast ? it % BROWS : it / 8;
                const int c = a.b_nfast ? it / BROWS : it % 8;
                if constexpr (CPLX) {
                    float x0[VPC], x1[VPC];  // rows 2j: (re, -im) ; 2j+1: (im, re)
#pragma unroll
                    for (int v = 0; v < CPC; ++v) {
                        const float re = R.b[i][2 * v] * fb, im = R.b[i][2 * v + 1] * fb;
                        x0[2 * v] = re;
                        x0[2 * v + 1] = -im;
                        x1[2 * v] = im;
                        x1[2 * v + 1] = re;
                    }
                    uint4 h0, l0, h1, l1;
                    if constexpr (BF16) {
                        Pack<true>::split8(x0, h0, l0);
                        Pack<true>::split8(x1, h1, l1);
                    } else {
                        Pack<false>::split4(x0, h0, l0, SPLIT);
                        Pack<false>::split4(x1, h1, l1, SPLIT);
                    }
                    *reinterpret_cast<uint4*>(sb + swz(2 * j, c)) = h0;
                    *reinterpret_cast<uint4*>(sb + swz(2 * j + 1, c)) = h1;
                    if constexpr (SPLIT) {
                        *reinterpret_cast<uint4*>(sb + kTileBytes + swz(2 * j, c)) = l0;
                        *reinterpret_cast<uint4*>(sb + kTileBytes + swz(2 * j + 1, c)) = l1;
                    }
                } else {
                    float x[VPC];
#pragma unroll
                    for (int v = 0; v < VPC; ++v) x[v] = R.b[i][v] * fb;
                    uint4 hi, lo;
                    if constexpr (BF16) Pack<true>::split8(x, hi, lo);
                    else Pack<false>::split4(x, hi, lo, SPLIT);
                    *reinterpret_cast<uint4*>(sb + swz(j, c)) = hi;
                    if constexpr (SPLIT) *reinterpret_cast<uint4*>(sb + kTileBytes + swz(j, c)) = lo;
                }
            }
            fence_proxy_async();
            mbar_arrive(&full_bar[s]);
            return true;
        };
        // two register sets: the gathers of k-block kb+1 are in flight while
        // k-block kb is converted and stored
        bool ok = true;
        Regs R0, R1;
        gather(0, R0);
        for (int kb = 0; kb < nkb && ok; kb += 2) {
            if (kb + 1 < nkb) gather(kb + 1, R1);
            if (!deposit(kb, R0)) {
                ok = false;
                break;
            }
            if (kb + 1 < nkb) {
                if (kb + 2 < nkb) gather(kb + 2, R0);
                if (!deposit(kb + 1, R1)) {
                    ok = false;
                    break;
                }
            }
        }
        if (!ok) abort_flag = 1;

        // ---------------- epilogue ----------------
        float lmax = 0.f;
        bool done = mbar_wait(&done_bar, 0u, &abort_flag);
        tc_fence_after();
        done = __all_sync(0xffffffffu, done && !abort_flag);  // tcgen05.ld is warp-collective
        if (done) {
            const int quad = warp & 3;                // TMEM lanes 32*quad.. belong to this warp
            const int row = quad * 32 + (tid & 31);   // TMEM lane = tile row
            const int64_t m = m0 + row;
            constexpr int kGroups = kProducers / 128;  // warps sharing a lane quadrant
            const int col0 = (warp >> 2) * (kBN / kGroups);
            for (int col = col0; col < col0 + kBN / kGroups; col += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)col, v);
                if (m < M) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        if (resid) v[i] = ldexpf(v[i], -resid);
                        lmax = fmaxf(lmax, fabsf(v[i]));
                    }
                    const int nfirst = CPLX ? col / 2 : col;
                    const int ncount = CPLX ? 8 : 16;
                    if (nfirst < nlim) {
                        float* crow = reinterpret_cast<float*>(Cinst) +
                                      ((b * M + m) * N + n0 + nfirst) * (CPLX ? 2 : 1);
                        if (nfirst + ncount <= nlim) {
#pragma unroll
                            for (int i = 0; i < 16; i += 4)
                                *reinterpret_cast<float4*>(crow + i) =
                                    make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                        } else {
                            const int vals = (nlim - nfirst) * (CPLX ? 2 : 1);
                            for (int i = 0; i < vals; ++i) crow[i] = v[i];
                        }
                    }
                }
            }
        } else {
            atomicExch(const_cast<int32_t*>(&a.ctl->status), (int32_t)TN_ETIMEOUT);
        }
        // block-free max over the producer warps
        for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        if ((tid & 31) == 0 && lmax > 0.f) atomicMax(sio.max_c, __float_as_uint(lmax));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        // the MMA thread committed done_bar after its last MMA (also on abort):
        // wait (bounded) for it so no MMA still writes the accumulator
        int dummy = 0;
        bool quiet = true;
        if ((tid & 31) == 0) quiet = mbar_wait(&done_bar, 0u, &dummy);
        quiet = __shfl_sync(0xffffffffu, quiet, 0);
        tc_fence_after();
        if (!quiet && (tid & 31) == 0) atomicExch(const_cast<int32_t*>(&a.ctl->status), (int32_t)TN_ETIMEOUT);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kBN));
    }
    if (a.t_done && tid == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        atomicMax(a.t_done, t);
    }
}

template <bool CPLX, int PREC>
static cudaError_t launch_tc_t(const TileArgs& a, cudaStream_t s) {
    constexpr int STAGES = PREC == 0 ? 4 : 3;
    constexpr int PARTS = PREC == 0 ? 1 : 2;
    constexpr int SMEM = STAGES * 2 * PARTS * kTileBytes + 1024;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_tc<CPLX, PREC, STAGES>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int64_t M = 1ll << a.nm, N = 1ll << a.nn;
    constexpr int NC = CPLX ? kBN / 2 : kBN;
    const int64_t tiles = ((M + kBM - 1) / kBM) * ((N + NC - 1) / NC);
    const int ni = a.in.n_inst > 1 ? a.in.n_inst : 1;
    dim3 grid((unsigned)tiles, 1, (unsigned)(a.nbatch * ni));
    k_tc<CPLX, PREC, STAGES><<<grid, kThreads, SMEM, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tc(const TileArgs& a, int prec, bool is_c, cudaStream_t s) {
    if (is_c) {
        if (prec == 0) return launch_tc_t<true, 0>(a, s);
        if (prec == 1) return launch_tc_t<true, 1>(a, s);
        return launch_tc_t<true, 2>(a, s);
    }
    if (prec == 0) return launch_tc_t<false, 0>(a, s);
    if (prec == 1) return launch_tc_t<false, 1>(a, s);
    return launch_tc_t<false, 2>(a, s);
}

}  // namespace tn
