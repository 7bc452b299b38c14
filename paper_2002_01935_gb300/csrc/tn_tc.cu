// tn_tc.cu -- tensor-core path for large nodes (tcgen05 + TMEM + TMA).
//
// A large tree node (Sec. 2 of arXiv 2002.01935: the inner product of two
// tensors over their shared labels) is a batched GEMM C[b] = A[b] B[b].
// It runs in three launches:
//   1. k_pack (row operand R) and 2. k_pack (column operand Q): a bit
//      permutation of the operand into K-major packed rows (TcGeom), staged
//      through shared memory so that both the read of the source layout and
//      the write of the packed layout are coalesced; the same pass applies
//      the slice offset of a sliced leaf, the power-of-two renormalisation,
//      the complex conjugation of the reverse sweep, the hi/lo split (TF32
//      round-to-nearest-away, or BF16 / FP16 round-to-nearest; FP16 after a
//      power-of-two shift into its range) and, for a complex Q,
//      the expansion into the rows (Re, -Im) and (Im, Re).
//   3. k_umma: a warp-specialised, persistent GEMM (one CTA per SM walking
//      the output tiles in grouped raster order).  One thread streams the
//      packed 16 KB tiles (128 rows x one 128-byte row of K, already laid
//      out in the 128-byte swizzle the UMMA descriptors expect) into a ring
//      of shared-memory stages with plain bulk copies (cp.async.bulk on the
//      TMA engine, one contiguous copy per tile and plane: the pack has
//      done the permutation, so no tensor map is needed); one thread issues
//      tcgen05.mma (kind::tf32, or kind::f16 with BF16 or FP16 operands)
//      into FP32 accumulators in tensor memory -- lo*hi, hi*lo, then hi*hi
//      for the split precisions -- rotating over up to four accumulators
//      along K; four (128-column tiles) or eight (256-column tiles)
//      epilogue warps drain each finished accumulator chain with
//      tcgen05.ld into FP32 registers, undo the residual scale, reduce the
//      node maximum and write C in the node's [batch][M][N] layout.
//      k_umma2 runs 256 x 256 tiles on CTA pairs (clusters of two, the
//      pair MMA tcgen05 cta_group::2, eight epilogue warps per CTA) when
//      the row tiles come in pairs; k_umma_planar (Re/Im planes) and
//      k_umma3m (three real products) are the other layouts.
// Complex nodes use one real GEMM with K doubled (4M): R holds interleaved
// (re, im) pairs along K and Q's expanded rows turn each accumulator column
// pair into (Re C, Im C).  The larger complex operand plays R (it is not
// expanded); when that is B the accumulator rows run over N and the
// epilogue writes the transpose.
// Every wait is bounded; on timeout the kernel records TN_ETIMEOUT in the
// control block, waits (bounded) for its copies and MMAs in flight, frees
// its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "../../include/tn.h"
#include "tn_internal.h"

namespace tn {

namespace {

constexpr int kBM = 128;              // accumulator rows (TMEM lanes) per tile
constexpr int kBN = 128;              // real accumulator columns per tile
constexpr int kRowBytes = 128;        // one swizzle row per stage and plane
constexpr int kTileBytes = kBM * kRowBytes;  // 16 KB per plane and operand
constexpr int kGemmThreads = 192;     // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int kNumAcc = 4;            // TMEM accumulators (128 columns each) in rotation
constexpr int kGroupRows = 32;        // row tiles per raster group (L2 reuse: R stays resident, Q streams)
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz
constexpr int kPackThreads = 256;
constexpr int kPackLow = 5;           // lowest bits of each order staged per tile
constexpr int kPackMaxTile = 1 << (2 * kPackLow);

// Pack CTAs for an operand of n entries: every CTA stages several 1024-entry
// tiles, so that its setup is amortised (measured: one tile per CTA made the
// packs of mid-size nodes slower, not faster).
inline unsigned pack_blocks(int64_t n, int ni) {
    (void)ni;
    return (unsigned)std::min<int64_t>(std::max<int64_t>(n / 8192, 1), (int64_t)sm_count() * 8);
}

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

// HALF: kind::f16 (BF16 or FP16 operands, the format is in idesc);
// otherwise kind::tf32.
template <bool HALF>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate) {
    if constexpr (HALF) {
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

// Add 32 accumulator columns (two x16 loads, one wait) into s[0..31].
__device__ __forceinline__ void tmem_add32(uint32_t taddr, float* s) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr + 16u));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) s[i] += __uint_as_float(r[i]);
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

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// One contiguous global -> shared bulk copy (TMA engine), completing on bar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Output stores of the GEMM epilogues: a node's final output is written once
// and read by a later launch step, so it is stored with the streaming
// (evict-first) hint and does not push the packed operands, which the other
// tiles of the node still read, out of L2; K-split partials, which the
// reduction reads right after, keep the normal policy.
__device__ __forceinline__ void st_out4(float* p, float4 v, bool stream) {
    if (stream) __stcs(reinterpret_cast<float4*>(p), v);
    else *reinterpret_cast<float4*>(p) = v;
}
__device__ __forceinline__ void st_out2(float* p, float2 v, bool stream) {
    if (stream) __stcs(reinterpret_cast<float2*>(p), v);
    else *reinterpret_cast<float2*>(p) = v;
}

// ---- CTA-pair helpers (k_umma2) ----
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Shared::cluster address of the object at local's offset in CTA `rank`.
__device__ __forceinline__ uint32_t peer_addr(const void* local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
    return r;
}

// Arrive (release, cluster scope) on a barrier given by its shared::cluster address.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// Bounded wait with cluster-scope acquire: the phase may have been completed
// by arrivals from the peer CTA.
__device__ __forceinline__ bool mbar_wait_cl(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    long long t0 = clock64();
    for (uint32_t i = 0;; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((i & 255) == 255) {
            if (*abort_flag) return false;
            if (clock64() - t0 > kWaitCycles) return false;
        }
    }
}

// One MMA of a CTA pair (M = 256 over the two CTAs' TMEM lanes; A rows and
// B columns split between the two CTAs' shared memory at the same offsets),
// issued by the even CTA.
template <bool HALF>
__device__ __forceinline__ void mma2(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t accumulate) {
    if constexpr (HALF) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
    }
}

// Arrive on the barrier at bar's offset in both CTAs of the pair once the
// pair MMAs issued so far have completed.
__device__ __forceinline__ void mma2_commit_both(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

// One packed element: the split parts of a value (TF32 keeps float bit
// patterns with the low 13 mantissa bits zero; BF16 is round to nearest).
template <int PREC>
struct Parts;
template <>
struct Parts<0> {
    using E = float;
    static __device__ __forceinline__ void split(float x, E& h, E& l) {
        h = to_tf32(x);
        l = 0.f;
    }
};
template <>
struct Parts<1> {
    using E = float;
    static __device__ __forceinline__ void split(float x, E& h, E& l) {
        h = to_tf32(x);
        l = to_tf32(x - h);
    }
};
template <>
struct Parts<3> : Parts<0> {};
template <>
struct Parts<2> {
    using E = __nv_bfloat16;
    static __device__ __forceinline__ void split(float x, E& h, E& l) {
        h = __float2bfloat16_rn(x);
        l = __float2bfloat16_rn(x - __bfloat162float(h));
    }
};
// FP16: the pack has already scaled x by 2^kF16Shift (|x| < 2^15)
template <>
struct Parts<4> {
    using E = __half;
    static __device__ __forceinline__ void split(float x, E& h, E& l) {
        h = __float2half_rn(x);
        l = __float2half_rn(x - __half2float(h));
    }
};

// 16-byte chunk position of (row, chunk) in a 128B-swizzled K-major tile
// (the layout of a TMA 128-byte swizzle and of the UMMA descriptors below).
__device__ __forceinline__ uint32_t swz(int row, int chunk) {
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

// Byte position of packed element (row, k) in a plane of 16 KB tiles
// (128 rows x one 128-byte swizzled row of K each, row tile by row tile,
// k-block by k-block within one).
__device__ __forceinline__ int64_t tile_pos(int64_t row, int64_t k, int64_t nkb, int lg_ke, int lg_esz) {
    const int64_t tile = (row >> 7) * nkb + (k >> lg_ke);
    const int byte = (int)(k & ((1 << lg_ke) - 1)) << lg_esz;
    return tile * kTileBytes + swz((int)(row & 127), byte >> 4) + (byte & 15);
}

// The same for the planar layout's 8 KB tiles: 128 rows x one 64-byte row
// of K in the 64-byte swizzle (16-byte chunk c of row r stored at chunk
// c ^ ((r >> 1) & 3); 8-row atoms of 512 bytes).
__device__ __forceinline__ uint32_t swz64(int row, int chunk) {
    return (uint32_t)((row >> 3) * 512 + (row & 7) * 64 + ((chunk ^ ((row >> 1) & 3)) << 4));
}

__device__ __forceinline__ int64_t tile_pos64(int64_t row, int64_t k, int64_t nkb, int lg_ke, int lg_esz) {
    const int64_t tile = (row >> 7) * nkb + (k >> lg_ke);
    const int byte = (int)(k & ((1 << lg_ke) - 1)) << lg_esz;
    return tile * (kTileBytes / 2) + swz64((int)(row & 127), byte >> 4) + (byte & 15);
}

// UMMA shared-memory descriptor for the planar tiles: K-major, 64-byte
// swizzle, 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc64(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;     // stride byte offset
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)4 << 61;              // SWIZZLE_64B
    return d;
}

// Write the packed elements (x, y) (adjacent along K) at byte position pos
// of the hi plane and of the lo plane lo_off bytes later.
template <int PREC>
__device__ __forceinline__ void put2(char* hi, int64_t lo_off, int64_t pos, float x, float y) {
    using P = Parts<PREC>;
    typename P::E hx, lx, hy, ly;
    P::split(x, hx, lx);
    P::split(y, hy, ly);
    if constexpr (PREC == 2) {
        __nv_bfloat162 h, l;
        h.x = hx; h.y = hy; l.x = lx; l.y = ly;
        *reinterpret_cast<__nv_bfloat162*>(hi + pos) = h;
        *reinterpret_cast<__nv_bfloat162*>(hi + lo_off + pos) = l;
    } else if constexpr (PREC == 4) {
        __half2 h, l;
        h.x = hx; h.y = hy; l.x = lx; l.y = ly;
        *reinterpret_cast<__half2*>(hi + pos) = h;
        *reinterpret_cast<__half2*>(hi + lo_off + pos) = l;
    } else {
        *reinterpret_cast<float2*>(hi + pos) = make_float2(hx, hy);
        if constexpr (PREC == 1) *reinterpret_cast<float2*>(hi + lo_off + pos) = make_float2(lx, ly);
    }
}

// Four adjacent packed elements (two K-adjacent complex entries of the 4M
// layout) in one store per plane: 8 bytes (16-bit formats) or 16 (TF32).
template <int PREC>
__device__ __forceinline__ void put4(char* hi, int64_t lo_off, int64_t pos, float a, float b, float c, float d) {
    if constexpr (PREC == 2 || PREC == 4) {
        // paired round-to-nearest conversions; the same parts as Parts<PREC>::split
        uint2 hv, lv;
        if constexpr (PREC == 4) {
            const __half2 h01 = __floats2half2_rn(a, b), h23 = __floats2half2_rn(c, d);
            const float2 f01 = __half22float2(h01), f23 = __half22float2(h23);
            const __half2 l01 = __floats2half2_rn(a - f01.x, b - f01.y);
            const __half2 l23 = __floats2half2_rn(c - f23.x, d - f23.y);
            hv = make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
            lv = make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
        } else {
            const __nv_bfloat162 h01 = __floats2bfloat162_rn(a, b), h23 = __floats2bfloat162_rn(c, d);
            const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
            const __nv_bfloat162 l01 = __floats2bfloat162_rn(a - f01.x, b - f01.y);
            const __nv_bfloat162 l23 = __floats2bfloat162_rn(c - f23.x, d - f23.y);
            hv = make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
            lv = make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
        }
        *reinterpret_cast<uint2*>(hi + pos) = hv;
        *reinterpret_cast<uint2*>(hi + lo_off + pos) = lv;
    } else {
        using P = Parts<PREC>;
        typename P::E h[4], l[4];
        P::split(a, h[0], l[0]);
        P::split(b, h[1], l[1]);
        P::split(c, h[2], l[2]);
        P::split(d, h[3], l[3]);
        *reinterpret_cast<float4*>(hi + pos) = make_float4(h[0], h[1], h[2], h[3]);
        if constexpr (PREC == 1) *reinterpret_cast<float4*>(hi + lo_off + pos) = make_float4(l[0], l[1], l[2], l[3]);
    }
}

template <int PREC>
__device__ __forceinline__ void put1(char* hi, int64_t lo_off, int64_t pos, float x) {
    using P = Parts<PREC>;
    typename P::E h, l;
    P::split(x, h, l);
    *reinterpret_cast<typename P::E*>(hi + pos) = h;
    if constexpr (PREC != 0) *reinterpret_cast<typename P::E*>(hi + lo_off + pos) = l;
}

}  // namespace

// ---------------------------------------------------------------------------
// k_pack: operand (role 0 = R, 1 = Q) -> packed K-major planes.
//
// Logical element index g (the packed order): K bits fastest, then the
// row/column bits of the operand, then the batch bits.  The source offset
// of g scatters each logical bit to the operand's own stride.  A tile is
// the set of logical bits holding the kPackLow lowest source strides and
// the kPackLow lowest packed positions; the remaining bits enumerate the
// tiles.  Each tile is read in source order (consecutive threads read
// consecutive source addresses), staged in shared memory, and written in
// packed order (consecutive threads write consecutive packed addresses).
// ---------------------------------------------------------------------------
template <bool CPLX, int PREC>
__global__ void __launch_bounds__(kPackThreads)
    k_pack(const __grid_constant__ TileArgs a, const __grid_constant__ PackPlan pr,
           const __grid_constant__ PackPlan pq, int blocks_r) {
    // blocks [0, blocks_r) pack R, the others Q (one launch for both operands)
    const int role = (int)blockIdx.x < blocks_r ? 0 : 1;
    const PackPlan& pp = role == 0 ? pr : pq;
    const int bx = role == 0 ? (int)blockIdx.x : (int)blockIdx.x - blocks_r;
    const int nbx = role == 0 ? blocks_r : (int)gridDim.x - blocks_r;
    using T = typename std::conditional<CPLX, float2, float>::type;
    __shared__ T stage[kPackMaxTile + kPackMaxTile / 32];  // +1 per 32: no bank conflicts
    __shared__ int64_t tsrc[kPackMaxTile];
    __shared__ int64_t tdst[kPackMaxTile];
    __shared__ uint16_t tidx[kPackMaxTile];

    const bool useB = (role == 0) == (a.tc_swap != 0);
    const int inst = blockIdx.y;
    const InstanceInfo& in = a.in;
    const int64_t slice = a.ctl->slice + (int64_t)inst * in.slice_step;
    if (slice >= a.ctl->slice_end) return;
    const int nk = a.nk;
    const TcGeom geo = tc_geom(a, CPLX, PREC);
    constexpr int LG_ESZ = (PREC == 2 || PREC == 4) ? 1 : 2, LG_KE = 7 - LG_ESZ;
    const int ESZ = CPLX ? 8 : 4;
    const T* src = reinterpret_cast<const T*>(useB ? a.B : a.A) +
                   (int64_t)inst * (useB ? in.b_is : in.a_is) +
                   slice_offset(useB ? a.slb : a.sla, slice);
    char* pk = reinterpret_cast<char*>(a.P) + (int64_t)inst * in.p_is * ESZ;
    char* hi = role == 0 ? pk : pk + geo.region_r;
    const int64_t lo_off = role == 0 ? geo.plane_r : geo.plane_q;
    const unsigned* mslot = useB ? a.sc.max_b : a.sc.max_a;
    if (mslot) mslot += (int64_t)inst * (useB ? in.sb_is : in.sa_is);
    const int e = exp_of(mslot);
    const float f = ldexpf(1.f, -max(-120, min(120, e)) + (PREC == 4 ? kF16Shift : 0));
    const bool conj = useB ? a.conj_b : a.conj_a;

    // the tile tables: source offset of each source-order index, packed
    // byte position and (padded) stage index of each packed-order index
    const int t = pp.t, u = pp.u;
    const int tsz = 1 << t;
    for (int i = threadIdx.x; i < tsz; i += blockDim.x) {
        int64_t so = 0, dg = 0;
        int idx = 0;
        for (int j = 0; j < t; ++j)
            if ((i >> j) & 1) {
                so += pp.src_add[j];
                dg ^= pp.dst_pos[j];
                idx += pp.idx_add[j];
            }
        tsrc[i] = so;
        tdst[i] = dg;
        tidx[i] = (uint16_t)(idx + (idx >> 5));
    }
    __syncthreads();
    const int64_t n_tiles = int64_t(1) << u;
    const int64_t K = int64_t(1) << nk;
    // tile bases by their bits, one bit per lane and a warp-wide sum (source
    // offset) and XOR (packed position); the loads of the next tile are
    // issued before the current one is written out (two tiles of reads in
    // flight)
    const int lane = threadIdx.x & 31;
    auto bases = [&](int64_t tile, int64_t& sb, int64_t& gb) {
        int64_t s0 = 0, g0 = 0;
        for (int j = lane; j < u; j += 32)
            if ((tile >> j) & 1) {
                s0 += pp.rest_src[j];
                g0 ^= pp.rest_pos[j];
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            g0 ^= __shfl_xor_sync(0xffffffffu, g0, o);
        }
        sb = s0;
        gb = g0;
    };
    constexpr int R = kPackMaxTile / kPackThreads;
    T ld[R];
    int64_t sb, gb;
    if ((int64_t)bx < n_tiles) {
        bases(bx, sb, gb);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = threadIdx.x + r * kPackThreads;
            if (i < tsz) ld[r] = src[sb + tsrc[i]];
        }
    }
    for (int64_t tile = bx; tile < n_tiles; tile += nbx) {
        const int64_t gb_cur = gb;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = threadIdx.x + r * kPackThreads;
            if (i < tsz) stage[i + (i >> 5)] = ld[r];
        }
        __syncthreads();
        const int64_t next = tile + nbx;
        if (next < n_tiles) {
            bases(next, sb, gb);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = threadIdx.x + r * kPackThreads;
                if (i < tsz) ld[r] = src[sb + tsrc[i]];
            }
        }
        const int64_t gbase = gb_cur;
        // two K-adjacent entries per thread (tile index bit 0 is K bit 0):
        // one store per plane for both
#pragma unroll
        for (int r = 0; r < kPackMaxTile / (2 * kPackThreads); ++r) {
            const int i = 2 * (threadIdx.x + r * kPackThreads);
            if (i >= tsz) break;
            const T v0 = stage[tidx[i]], v1 = stage[tidx[i + 1]];
            const int64_t pos = gbase ^ tdst[i];  // byte position of the first entry (even k)
            if constexpr (CPLX && PREC == 3) {
                // 3M: planes Re, Im, Re + Im of either operand, K not doubled
                const float re0 = v0.x * f, im0 = (conj ? -v0.y : v0.y) * f;
                const float re1 = v1.x * f, im1 = (conj ? -v1.y : v1.y) * f;
                put2<0>(hi, 0, pos, re0, re1);
                put2<0>(hi + lo_off, 0, pos, im0, im1);
                put2<0>(hi + 2 * lo_off, 0, pos, re0 + im0, re1 + im1);
            } else if constexpr (CPLX) {
                const float re0 = v0.x * f, im0 = (conj ? -v0.y : v0.y) * f;
                const float re1 = v1.x * f, im1 = (conj ? -v1.y : v1.y) * f;
                if (geo.planar) {
                    // planes Re hi, Re lo, Im hi, Im lo of either operand
                    put2<PREC>(hi, lo_off, pos, re0, re1);
                    put2<PREC>(hi + 2 * lo_off, lo_off, pos, im0, im1);
                } else if (role == 0) {
                    put4<PREC>(hi, lo_off, pos, re0, im0, re1, im1);
                } else {
                    put4<PREC>(hi, lo_off, pos, re0, -im0, re1, -im1);
                    put4<PREC>(hi, lo_off, pos ^ pp.pos_row1, im0, re0, im1, re1);
                }
            } else {
                put2<PREC>(hi, lo_off, pos, v0 * f, v1 * f);
            }
        }
        __syncthreads();
    }
}

// k-blocks per TMEM accumulator chain before the epilogue adds it into FP32
// registers.  Each hand-off costs a round trip between the MMA thread and
// the epilogue (and a drain of the accumulator), so longer chains keep the
// tensor pipe busier, while every extra k-block in a chain adds the tensor
// core's own accumulation rounding.  Measured on the 7x7x14 amplitude (split
// products issued small-first, see the MMA loops): chains of 2 take the
// slice 10% faster than chains of 1 and keep its FP16-split error against
// the oracle at 3.6e-6 (every sub-slice within 4.9e-6).
__host__ __device__ constexpr int umma_chain(int prec) { return prec == 0 ? 4 : 2; }

// ---------------------------------------------------------------------------
// k_umma: bulk-copy-fed tcgen05 GEMM over the packed planes, persistent: the
// work items (output tile in grouped raster order, K part, batch entry and
// instance; tile fastest) are dealt to the CTAs round robin, one CTA per SM.
// The copy thread, the MMA thread and the epilogue warps each walk the same
// item sequence; the stage ring and the accumulator rotation run on across
// items, so the next item's copies and first MMAs overlap this item's final
// drain and output stores, and no CTA is launched or torn down per tile.
// ---------------------------------------------------------------------------
struct UmmaItem {
    int tm, tn, sp;
    int64_t b;
    int inst;
    bool live;
};

__device__ __forceinline__ UmmaItem umma_item(int64_t w, int tiles_m, int tiles_n, int nsplit,
                                              int64_t nbatch, int64_t slice0, int64_t slice_step,
                                              int64_t slice_end, int group_rows) {
    UmmaItem it;
    const int64_t tiles = (int64_t)tiles_m * tiles_n;
    const int x = (int)(w % tiles);
    const int64_t rest = w / tiles;
    it.sp = (int)(rest % nsplit);
    const int64_t z = rest / nsplit;
    it.b = z % nbatch;
    it.inst = (int)(z / nbatch);
    // grouped raster: group_rows row tiles share the column tiles they stream
    const int per_group = group_rows * tiles_n;
    const int grp = x / per_group;
    const int first = grp * group_rows;
    const int gsz = min(group_rows, tiles_m - first);
    const int r = x - grp * per_group;
    it.tm = first + r % gsz;
    it.tn = r / gsz;
    it.live = slice0 + (int64_t)it.inst * slice_step < slice_end;
    return it;
}

template <bool CPLX, int PREC, int STAGES, int BN>
__global__ void __launch_bounds__(64 + BN, 1)
    k_umma(const __grid_constant__ TileArgs a, int nacc, int grp_rows) {
    constexpr bool HALF = PREC == 2 || PREC == 4;   // 16-bit operands, kind::f16
    constexpr bool SPLIT = PREC != 0;
    constexpr int PARTS = SPLIT ? 2 : 1;
    constexpr int QB = BN * kRowBytes;                    // one Q part per stage
    constexpr int QT = BN / kBM;                           // packed 128-row Q tiles per part
    constexpr int EPI_WARPS = BN / 32;                     // 128 rows x BN columns, 128 each
    constexpr int STAGE_BYTES = PARTS * (kTileBytes + QB);
    constexpr int KE = HALF ? 64 : 32;     // packed elements per 128-byte row
    constexpr int MMA_K = HALF ? 16 : 8;   // K per instruction
    constexpr int KSTEPS = KE / MMA_K;
    constexpr uint32_t FMT = PREC == 2 ? 1u : (PREC == 4 ? 0u : 2u);  // BF16, FP16, TF32

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
    __shared__ uint64_t acc_full[kNumAcc], acc_empty[kNumAcc];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ int consumed;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int nsplit = a.split > 1 ? a.split : 1;
    // two-level accumulation: a chain of `chain` k-blocks accumulates in one
    // TMEM accumulator; the epilogue warps add every finished chain into FP32
    // registers (round to nearest), which keeps the tensor-core adder's long
    // accumulation error out of the result
    const int chain = umma_chain(PREC);
    const InstanceInfo& in = a.in;
    const int ni = in.n_inst > 1 ? in.n_inst : 1;
    const int64_t slice0 = a.ctl->slice, slice_end = a.ctl->slice_end;
    const TcGeom geo = tc_geom(a, CPLX, PREC);
    const int nkl = (int)(geo.nkb / nsplit);   // k-blocks of one K part
    const int tiles_m = (int)(geo.rows_r / kBM), tiles_n = (int)(geo.cols_q / BN);
    const int64_t n_items = (int64_t)tiles_m * tiles_n * nsplit * a.nbatch * ni;
    const int nchain = (nkl + chain - 1) / chain;
    const int acc_cols = nacc * BN;
    const uint32_t alloc_cols = acc_cols <= 128 ? 128u : (acc_cols <= 256 ? 256u : 512u);
    const int ESZ = CPLX ? 8 : 4;
    const int64_t M = int64_t(1) << a.nm, N = int64_t(1) << a.nn;
#define UMMA_ITEM(w) umma_item((w), tiles_m, tiles_n, nsplit, a.nbatch, slice0, in.slice_step, slice_end, grp_rows)

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        for (int q = 0; q < kNumAcc; ++q) {
            mbar_init(&acc_full[q], 1);
            mbar_init(&acc_empty[q], EPI_WARPS);  // one arrival per epilogue warp
        }
        abort_flag = 0;
        consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(alloc_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ---------------- bulk-copy producer ----------------
        if (tid == 0) {
            int issued = 0;  // k-blocks over all items (stage ring position)
            for (int64_t w = blockIdx.x; w < n_items && !*(volatile int*)&abort_flag; w += gridDim.x) {
                const UmmaItem it = UMMA_ITEM(w);
                if (!it.live) continue;
                const char* pk = reinterpret_cast<const char*>(a.P) + (int64_t)it.inst * in.p_is * ESZ;
                const int64_t kb0 = (int64_t)it.sp * nkl;
                const char* r_src = pk + ((it.b * tiles_m + it.tm) * geo.nkb + kb0) * kTileBytes;
                const char* q_src = pk + geo.region_r + ((it.b * tiles_n + it.tn) * QT * geo.nkb + kb0) * kTileBytes;
                for (int j = 0; j < nkl; ++j) {
                    const int s = issued % STAGES;
                    if (issued >= STAGES &&
                        !mbar_wait(&empty_bar[s], (uint32_t)(((issued / STAGES) + 1) & 1), &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    uint8_t* st = smem + s * STAGE_BYTES;
                    mbar_expect_tx(&full_bar[s], STAGE_BYTES);
                    const int64_t o = (int64_t)j * kTileBytes;
                    bulk_load(st, r_src + o, kTileBytes, &full_bar[s]);
                    if constexpr (SPLIT) bulk_load(st + kTileBytes, r_src + geo.plane_r + o, kTileBytes, &full_bar[s]);
                    uint8_t* sq = st + PARTS * kTileBytes;
                    // BN columns: QT consecutive 128-row packed tiles, one after the other in smem
#pragma unroll
                    for (int h = 0; h < QT; ++h) {
                        const int64_t oh = o + (int64_t)h * geo.nkb * kTileBytes;
                        bulk_load(sq + h * kTileBytes, q_src + oh, kTileBytes, &full_bar[s]);
                        if constexpr (SPLIT)
                            bulk_load(sq + QB + h * kTileBytes, q_src + geo.plane_q + oh, kTileBytes, &full_bar[s]);
                    }
                    ++issued;
                }
            }
            if (abort_flag) {
                // wait (bounded) for the copies still in flight before leaving
                int dummy = 0;
                for (int j = *(volatile int*)&consumed; j < issued; ++j)
                    mbar_wait(&full_bar[j % STAGES], (uint32_t)((j / STAGES) & 1), &dummy);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (tid == 32) {
            const uint32_t idesc = instr_desc(FMT, kBM, BN);
            int gj = 0, gc = 0;  // k-blocks and chains over all items
            for (int64_t w = blockIdx.x; w < n_items && !*(volatile int*)&abort_flag; w += gridDim.x) {
                if (!UMMA_ITEM(w).live) continue;
                int q = 0;
                for (int j = 0; j < nkl; ++j, ++gj) {
                    const int s = gj % STAGES;
                    if (!mbar_wait(&full_bar[s], (uint32_t)((gj / STAGES) & 1), &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    const bool first = j % chain == 0;
                    if (first) {
                        // a chain reuses accumulator q once the epilogue has drained it
                        q = gc % nacc;
                        if (gc >= nacc &&
                            !mbar_wait(&acc_empty[q], (uint32_t)(((gc / nacc) + 1) & 1), &abort_flag)) {
                            abort_flag = 1;
                            break;
                        }
                    }
                    tc_fence_after();
                    const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
                    const uint32_t r_hi = base, q_hi = base + PARTS * kTileBytes;
                    const uint32_t r_lo = base + kTileBytes, q_lo = q_hi + QB;
                    const uint32_t d = tmem + (uint32_t)(q * BN);
                    // split precisions: the small hi*lo and lo*hi products first, the
                    // large hi*hi products last, so that the small ones are not added
                    // into an accumulator already holding the large sum (the tensor
                    // core's adder drops bits relative to the larger operand)
                    if constexpr (SPLIT) {
#pragma unroll
                        for (int k = 0; k < KSTEPS; ++k) {
                            const uint32_t off = k * MMA_K * (HALF ? 2 : 4);
                            mma<HALF>(d, smem_desc(r_hi + off), smem_desc(q_lo + off), idesc,
                                       (!first || k > 0) ? 1u : 0u);
                            mma<HALF>(d, smem_desc(r_lo + off), smem_desc(q_hi + off), idesc, 1u);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < KSTEPS; ++k) {
                        const uint32_t off = k * MMA_K * (HALF ? 2 : 4);
                        const uint32_t acc0 = (SPLIT || !first || k > 0) ? 1u : 0u;
                        mma<HALF>(d, smem_desc(r_hi + off), smem_desc(q_hi + off), idesc, acc0);
                    }
                    mma_commit(&empty_bar[s]);
                    if (j % chain == chain - 1 || j == nkl - 1) {
                        mma_commit(&acc_full[q]);
                        ++gc;
                    }
                    *(volatile int*)&consumed = gj + 1;
                }
            }
            mma_commit(&done_bar);  // arrives once every MMA issued above has completed
        }
    } else {
        // ---------------- epilogue (warps 2..) ----------------
        const int quad = warp & 3;                   // TMEM lanes 32*quad.. belong to this warp
        const int cbase = ((warp - 2) >> 2) * kBM;   // this warp's 128 of the BN columns
        float sum[kBM];
        bool ok = true;
        int gc = 0;  // chains over all items
        for (int64_t w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
            const UmmaItem it = UMMA_ITEM(w);
            if (!it.live) continue;
            // renormalisation: the pack applied 2^-clamp(e); the rest is undone here
            ScaleIO sio = a.sc;
            if (sio.max_a) sio.max_a += (int64_t)it.inst * in.sa_is;
            if (sio.exp_a) sio.exp_a += (int64_t)it.inst * in.sa_is;
            if (sio.max_b) sio.max_b += (int64_t)it.inst * in.sb_is;
            if (sio.exp_b) sio.exp_b += (int64_t)it.inst * in.sb_is;
            sio.max_c += (int64_t)it.inst * in.sc_is;
            sio.exp_c += (int64_t)it.inst * in.sc_is;
            const int eA = exp_of(sio.max_a), eB = exp_of(sio.max_b);
            const int resid = (eA - max(-120, min(120, eA))) + (eB - max(-120, min(120, eB))) +
                              (PREC == 4 ? 2 * kF16Shift : 0);
            if (it.tm == 0 && it.tn == 0 && it.sp == 0 && it.b == 0 && tid == 64 && sio.exp_c)
                *sio.exp_c = (sio.exp_a ? *sio.exp_a : 0) + (sio.exp_b ? *sio.exp_b : 0) + eA + eB;
#pragma unroll
            for (int i = 0; i < kBM; ++i) sum[i] = 0.f;
            for (int ch = 0; ch < nchain; ++ch, ++gc) {
                const int q = gc % nacc;
                const bool got = mbar_wait(&acc_full[q], (uint32_t)((gc / nacc) & 1), &abort_flag);
                ok = __all_sync(0xffffffffu, got && !abort_flag);  // tcgen05.ld is warp-collective
                if (!ok) break;
                tc_fence_after();
                const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(q * BN + cbase);
#pragma unroll
                for (int col = 0; col < kBM; col += 32) tmem_add32(ta + (uint32_t)col, sum + col);
                tc_fence_before();
                __syncwarp();
                if ((tid & 31) == 0) mbar_arrive(&acc_empty[q]);
            }
            if (!ok) break;
            float lmax = 0.f;
            const int row = it.tm * kBM + quad * 32 + (tid & 31);
            const int col0 = it.tn * BN;
            const int64_t b = it.b;
            // the node's output, or this part's FP32 partial product (same layout)
            float* C = nsplit > 1
                           ? reinterpret_cast<float*>(reinterpret_cast<char*>(a.P) +
                                                      (int64_t)it.inst * in.p_is * ESZ + geo.part_off) +
                                 (int64_t)it.sp * a.nbatch * M * N * (CPLX ? 2 : 1)
                           : reinterpret_cast<float*>(a.C) + (int64_t)it.inst * in.c_is * (CPLX ? 2 : 1);
            const int rs = nsplit > 1 ? 0 : resid;
#pragma unroll
            for (int cc = 0; cc < kBM; cc += 16) {
                float* v = sum + cc;
                const int col = cbase + cc;
                if (col0 + col >= geo.cols_valid) continue;  // padding columns of a narrow node
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    if (rs) v[i] = ldexpf(v[i], -rs);
                    lmax = fmaxf(lmax, fabsf(v[i]));
                }
                if constexpr (CPLX) {
                    const int64_t j0 = (col0 + col) / 2;  // first complex column of the chunk
                    if (!a.tc_swap) {
                        float* crow = C + ((b * M + row) * N + j0) * 2;
#pragma unroll
                        for (int i = 0; i < 16; i += 4)
                            st_out4(crow + i, make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]), nsplit == 1);
                    } else {
                        // rows run over N, complex columns over M
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            st_out2(C + ((b * M + j0 + i) * N + row) * 2, make_float2(v[2 * i], v[2 * i + 1]),
                                        nsplit == 1);
                    }
                } else {
                    float* crow = C + (b * M + row) * N + col0 + col;
#pragma unroll
                    for (int i = 0; i < 16; i += 4)
                        st_out4(crow + i, make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]), nsplit == 1);
                }
            }
            if (nsplit == 1) {
                for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
                if ((tid & 31) == 0 && lmax > 0.f) atomicMax(sio.max_c, __float_as_uint(lmax));
            }
        }
        if (!ok && (tid & 31) == 0) atomicExch(const_cast<int32_t*>(&a.ctl->status), (int32_t)TN_ETIMEOUT);
    }
#undef UMMA_ITEM
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        // no MMA may still write the accumulators when they are freed
        int dummy = 0;
        bool quiet = true;
        if (tid == 32) quiet = mbar_wait(&done_bar, 0u, &dummy);
        quiet = __shfl_sync(0xffffffffu, quiet, 0);
        tc_fence_after();
        if (!quiet && tid == 32) atomicExch(const_cast<int32_t*>(&a.ctl->status), (int32_t)TN_ETIMEOUT);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(alloc_cols));
    }
    if (a.t_done && tid == 0 && nsplit == 1) {
        unsigned long long tnow;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(tnow));
        atomicMax(a.t_done, tnow);
    }
}

// ---------------------------------------------------------------------------
// k_umma2: the persistent GEMM on CTA pairs (clusters of two, one CTA per
// SM) with the pair MMA (tcgen05 cta_group::2): a pair computes a 256-row x
// 256-column tile, each CTA holding its own 128 rows of R and one of the two
// 128-row tiles of Q in its shared memory, and its own 128 accumulator rows
// in its tensor memory.  Per k-block an SM thus receives 64 KB of operands
// (FP16 / BF16 / TF32 split) instead of the 96 KB of a single-CTA 128 x 256
// tile, and three stages fit in its shared memory.  Pair item v is the work
// items 2v (even CTA: row tile tm, Q tile 0) and 2v + 1 (odd CTA: row tile
// tm + 1, Q tile 1) of k_umma's item order.
// Synchronisation: each CTA's copy thread fills its own stage and barrier;
// the odd CTA's relay thread forwards each completed stage to the even
// CTA's full barrier (two arrivals per phase); the even CTA's MMA thread
// issues the pair MMAs and commits to the empty, accumulator-full and done
// barriers of both CTAs; the epilogue warps of both CTAs arrive on the even
// CTA's accumulator-empty barriers.  Tensor memory is allocated and freed
// by one warp of each CTA together.
// ---------------------------------------------------------------------------
template <bool CPLX, int PREC, int STAGES, int BN>
__global__ void __launch_bounds__(320, 1)
    k_umma2(const __grid_constant__ TileArgs a, int nacc, int grp_rows) {
    // BN: pair tile columns, 256 or 128; each CTA holds BN / 2 Q rows
    constexpr bool HALF = PREC == 2 || PREC == 4;
    constexpr bool SPLIT = PREC != 0;
    constexpr int PARTS = SPLIT ? 2 : 1;
    constexpr int QT = BN / kBM;                            // packed Q tiles per pair tile
    constexpr int QHB = BN / 2 * kRowBytes;                // this CTA's Q rows, per part
    constexpr int EPI_WARPS = 8;
    constexpr int ECOLS = BN / 2;                          // accumulator columns per epilogue warp
    constexpr int STAGE_BYTES = PARTS * (kTileBytes + QHB);
    constexpr int KE = HALF ? 64 : 32;
    constexpr int MMA_K = HALF ? 16 : 8;
    constexpr int KSTEPS = KE / MMA_K;
    constexpr uint32_t FMT = PREC == 2 ? 1u : (PREC == 4 ? 0u : 2u);

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
    __shared__ uint64_t acc_full[kNumAcc], acc_empty[kNumAcc];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ int consumed;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int nsplit = a.split > 1 ? a.split : 1;
    const int chain = umma_chain(PREC);   // k-blocks per accumulator chain (see k_umma)
    const InstanceInfo& in = a.in;
    const int ni = in.n_inst > 1 ? in.n_inst : 1;
    const int64_t slice0 = a.ctl->slice, slice_end = a.ctl->slice_end;
    const TcGeom geo = tc_geom(a, CPLX, PREC);
    const int nkl = (int)(geo.nkb / nsplit);
    const int tiles_m = (int)(geo.rows_r / kBM), tiles_n = (int)(geo.cols_q / BN);
    const int64_t n_pairs = (int64_t)tiles_m * tiles_n * nsplit * a.nbatch * ni / 2;
    const int nchain = (nkl + chain - 1) / chain;
    const uint32_t alloc_cols = nacc * BN <= 128 ? 128u : (nacc * BN <= 256 ? 256u : 512u);
    const int ESZ = CPLX ? 8 : 4;
    const int64_t M = int64_t(1) << a.nm, N = int64_t(1) << a.nn;
    const int64_t v0 = blockIdx.x >> 1, vstep = gridDim.x >> 1;
#define UMMA2_ITEM(v) \
    umma_item(2 * (v) + rank, tiles_m, tiles_n, nsplit, a.nbatch, slice0, in.slice_step, slice_end, grp_rows)

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            // even CTA: its own copies' arrival + the odd CTA's relay
            mbar_init(&full_bar[s], leader ? 2 : 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        for (int q = 0; q < kNumAcc; ++q) {
            mbar_init(&acc_full[q], 1);
            mbar_init(&acc_empty[q], 2 * EPI_WARPS);  // both CTAs' epilogue warps (even CTA's copy used)
        }
        abort_flag = 0;
        consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    // the peer's arrivals, copies and commits may only come once its barriers exist
    cluster_sync();
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(alloc_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ---------------- bulk-copy producer (both CTAs, own stages) ----------------
        if (tid == 0) {
            int issued = 0;
            for (int64_t v = v0; v < n_pairs && !*(volatile int*)&abort_flag; v += vstep) {
                const UmmaItem it = UMMA2_ITEM(v);
                if (!it.live) continue;
                const char* pk = reinterpret_cast<const char*>(a.P) + (int64_t)it.inst * in.p_is * ESZ;
                const int64_t kb0 = (int64_t)it.sp * nkl;
                const char* r_src = pk + ((it.b * tiles_m + it.tm) * geo.nkb + kb0) * kTileBytes;
                // this CTA's half of the pair's Q rows: Q tile `rank` (BN 256), or
                // rows 64 rank .. 64 rank + 63 of the Q tile (BN 128)
                const char* q_src = pk + geo.region_r +
                                    (QT == 2 ? (((it.b * tiles_n + it.tn) * QT + rank) * geo.nkb + kb0) * kTileBytes
                                             : ((it.b * tiles_n + it.tn) * geo.nkb + kb0) * kTileBytes + rank * QHB);
                for (int j = 0; j < nkl; ++j) {
                    const int s = issued % STAGES;
                    if (issued >= STAGES &&
                        !mbar_wait_cl(&empty_bar[s], (uint32_t)(((issued / STAGES) + 1) & 1), &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    uint8_t* st = smem + s * STAGE_BYTES;
                    mbar_expect_tx(&full_bar[s], STAGE_BYTES);
                    const int64_t o = (int64_t)j * kTileBytes;
                    // stage: R hi, Q hi, R lo, Q lo
                    bulk_load(st, r_src + o, kTileBytes, &full_bar[s]);
                    bulk_load(st + kTileBytes, q_src + o, QHB, &full_bar[s]);
                    if constexpr (SPLIT) {
                        bulk_load(st + kTileBytes + QHB, r_src + geo.plane_r + o, kTileBytes, &full_bar[s]);
                        bulk_load(st + 2 * kTileBytes + QHB, q_src + geo.plane_q + o, QHB, &full_bar[s]);
                    }
                    ++issued;
                }
            }
            if (*(volatile int*)&abort_flag) {
                // wait (bounded) for this CTA's copies still in flight before leaving
                int dummy = 0;
                for (int j = *(volatile int*)&consumed; j < issued; ++j)
                    mbar_wait(&full_bar[j % STAGES], (uint32_t)((j / STAGES) & 1), &dummy);
            }
        }
    } else if (warp == 1) {
        if (tid == 32 && leader) {
            // ---------------- pair MMA issuer (even CTA) ----------------
            const uint32_t idesc = instr_desc(FMT, 2 * kBM, BN);
            int gj = 0, gc = 0;
            for (int64_t v = v0; v < n_pairs && !*(volatile int*)&abort_flag; v += vstep) {
                if (!UMMA2_ITEM(v).live) continue;
                int q = 0;
                for (int j = 0; j < nkl; ++j, ++gj) {
                    const int s = gj % STAGES;
                    if (!mbar_wait_cl(&full_bar[s], (uint32_t)((gj / STAGES) & 1), &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    const bool first = j % chain == 0;
                    if (first) {
                        q = gc % nacc;
                        if (gc >= nacc &&
                            !mbar_wait_cl(&acc_empty[q], (uint32_t)(((gc / nacc) + 1) & 1), &abort_flag)) {
                            abort_flag = 1;
                            break;
                        }
                    }
                    tc_fence_after();
                    const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
                    const uint32_t r_hi = base, q_hi = base + kTileBytes;
                    const uint32_t r_lo = base + kTileBytes + QHB, q_lo = base + 2 * kTileBytes + QHB;
                    const uint32_t d = tmem + (uint32_t)(q * BN);
                    // split precisions: the small hi*lo and lo*hi products first, the
                    // large hi*hi products last, so that the small ones are not added
                    // into an accumulator already holding the large sum (the tensor
                    // core's adder drops bits relative to the larger operand)
                    if constexpr (SPLIT) {
#pragma unroll
                        for (int k = 0; k < KSTEPS; ++k) {
                            const uint32_t off = k * MMA_K * (HALF ? 2 : 4);
                            mma2<HALF>(d, smem_desc(r_hi + off), smem_desc(q_lo + off), idesc,
                                       (!first || k > 0) ? 1u : 0u);
                            mma2<HALF>(d, smem_desc(r_lo + off), smem_desc(q_hi + off), idesc, 1u);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < KSTEPS; ++k) {
                        const uint32_t off = k * MMA_K * (HALF ? 2 : 4);
                        const uint32_t acc0 = (SPLIT || !first || k > 0) ? 1u : 0u;
                        mma2<HALF>(d, smem_desc(r_hi + off), smem_desc(q_hi + off), idesc, acc0);
                    }
                    mma2_commit_both(&empty_bar[s]);
                    if (j % chain == chain - 1 || j == nkl - 1) {
                        mma2_commit_both(&acc_full[q]);
                        ++gc;
                    }
                    *(volatile int*)&consumed = gj + 1;
                }
            }
            mma2_commit_both(&done_bar);  // both CTAs: every pair MMA issued above has completed
        } else if (tid == 32) {
            // ---------------- relay (odd CTA): own stage complete -> even CTA's full barrier ----------------
            int gj = 0;
            for (int64_t v = v0; v < n_pairs && !*(volatile int*)&abort_flag; v += vstep) {
                if (!UMMA2_ITEM(v).live) continue;
                for (int j = 0; j < nkl; ++j, ++gj) {
                    const int s = gj % STAGES;
                    if (!mbar_wait(&full_bar[s], (uint32_t)((gj / STAGES) & 1), &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    mbar_arrive_cluster(peer_addr(&full_bar[s], 0));
                    *(volatile int*)&consumed = gj + 1;
                }
            }
        }
    } else {
        // ---------------- epilogue (warps 2..9 of both CTAs, own TMEM lanes) ----------------
        const int quad = warp & 3;
        const int cbase = ((warp - 2) >> 2) * ECOLS;
        float sum[ECOLS];
        bool ok = true;
        int gc = 0;
        for (int64_t v = v0; v < n_pairs && ok; v += vstep) {
            const UmmaItem it = UMMA2_ITEM(v);
            if (!it.live) continue;
            ScaleIO sio = a.sc;
            if (sio.max_a) sio.max_a += (int64_t)it.inst * in.sa_is;
            if (sio.exp_a) sio.exp_a += (int64_t)it.inst * in.sa_is;
            if (sio.max_b) sio.max_b += (int64_t)it.inst * in.sb_is;
            if (sio.exp_b) sio.exp_b += (int64_t)it.inst * in.sb_is;
            sio.max_c += (int64_t)it.inst * in.sc_is;
            sio.exp_c += (int64_t)it.inst * in.sc_is;
            const int eA = exp_of(sio.max_a), eB = exp_of(sio.max_b);
            const int resid = (eA - max(-120, min(120, eA))) + (eB - max(-120, min(120, eB))) +
                              (PREC == 4 ? 2 * kF16Shift : 0);
            if (it.tm == 0 && it.tn == 0 && it.sp == 0 && it.b == 0 && tid == 64 && sio.exp_c)
                *sio.exp_c = (sio.exp_a ? *sio.exp_a : 0) + (sio.exp_b ? *sio.exp_b : 0) + eA + eB;
#pragma unroll
            for (int i = 0; i < ECOLS; ++i) sum[i] = 0.f;
            for (int ch = 0; ch < nchain; ++ch, ++gc) {
                const int q = gc % nacc;
                const bool got = mbar_wait_cl(&acc_full[q], (uint32_t)((gc / nacc) & 1), &abort_flag);
                ok = __all_sync(0xffffffffu, got && !abort_flag);
                if (!ok) break;
                tc_fence_after();
                const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(q * BN + cbase);
#pragma unroll
                for (int col = 0; col < ECOLS; col += 32) tmem_add32(ta + (uint32_t)col, sum + col);
                tc_fence_before();
                __syncwarp();
                if ((tid & 31) == 0) {
                    if (leader) mbar_arrive(&acc_empty[q]);
                    else mbar_arrive_cluster(peer_addr(&acc_empty[q], 0));
                }
            }
            if (!ok) break;
            float lmax = 0.f;
            const int row = it.tm * kBM + quad * 32 + (tid & 31);
            const int col0 = it.tn * BN;
            const int64_t b = it.b;
            float* C = nsplit > 1
                           ? reinterpret_cast<float*>(reinterpret_cast<char*>(a.P) +
                                                      (int64_t)it.inst * in.p_is * ESZ + geo.part_off) +
                                 (int64_t)it.sp * a.nbatch * M * N * (CPLX ? 2 : 1)
                           : reinterpret_cast<float*>(a.C) + (int64_t)it.inst * in.c_is * (CPLX ? 2 : 1);
            const int rs = nsplit > 1 ? 0 : resid;
#pragma unroll
            for (int cc = 0; cc < ECOLS; cc += 16) {
                float* w = sum + cc;
                const int col = cbase + cc;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    if (rs) w[i] = ldexpf(w[i], -rs);
                    lmax = fmaxf(lmax, fabsf(w[i]));
                }
                if constexpr (CPLX) {
                    const int64_t j0 = (col0 + col) / 2;
                    if (!a.tc_swap) {
                        float* crow = C + ((b * M + row) * N + j0) * 2;
#pragma unroll
                        for (int i = 0; i < 16; i += 4)
                            st_out4(crow + i, make_float4(w[i], w[i + 1], w[i + 2], w[i + 3]), nsplit == 1);
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            st_out2(C + ((b * M + j0 + i) * N + row) * 2, make_float2(w[2 * i], w[2 * i + 1]),
                                        nsplit == 1);
                    }
                } else {
                    float* crow = C + (b * M + row) * N + col0 + col;
#pragma unroll
                    for (int i = 0; i < 16; i += 4)
                        st_out4(crow + i, make_float4(w[i], w[i + 1], w[i + 2], w[i + 3]), nsplit == 1);
                }
            }
            if (nsplit == 1) {
                for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
                if ((tid & 31) == 0 && lmax > 0.f) atomicMax(sio.max_c, __float_as_uint(lmax));
            }
        }
        if (!ok && (tid & 31) == 0) atomicExch(const_cast<int32_t*>(&a.ctl->status), (int32_t)TN_ETIMEOUT);
    }
#undef UMMA2_ITEM
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        // no pair MMA may still write either CTA's accumulators when they are freed
        int dummy = 0;
        bool quiet = true;
        if (tid == 32) quiet = mbar_wait_cl(&done_bar, 0u, &dummy);
        quiet = __shfl_sync(0xffffffffu, quiet, 0);
        tc_fence_after();
        if (!quiet && tid == 32) atomicExch(const_cast<int32_t*>(&a.ctl->status), (int32_t)TN_ETIMEOUT);
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(alloc_cols));
    }
    if (a.t_done && tid == 0 && nsplit == 1) {
        unsigned long long tnow;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(tnow));
        atomicMax(a.t_done, tnow);
    }
    // neither CTA leaves while the other may still arrive on its barriers
    cluster_sync();
}

// ---------------------------------------------------------------------------
// k_umma_planar: complex node in a split precision over the planar layout.
// A tile is 128 complex rows x 128 complex columns; each stage holds one
// 64-byte K row of the four planes of R and of Q (8 KB each).  Per K step
// the MMA thread issues the three split products of Re R Re Q and of
// Im R Im Q (negated) into the Re C accumulator and of Re R Im Q and Im R
// Re Q into the Im C accumulator; the accumulator pair rotates between two
// TMEM halves along K, and the eight epilogue warps drain each finished pair
// into FP32 registers as k_umma does.  blockIdx.x: output tile (grouped
// raster), y: K split, z: batch entry and instance.
// ---------------------------------------------------------------------------
template <int PREC, int STAGES>
__global__ void __launch_bounds__(320, 1)
    k_umma_planar(const __grid_constant__ TileArgs a) {
    constexpr bool HALF = PREC == 2 || PREC == 4;
    constexpr int PT = kTileBytes / 2;                   // 8 KB: one plane of one operand
    constexpr int STAGE_BYTES = 8 * PT;                  // 4 planes of R, 4 of Q
    constexpr int MMA_K = HALF ? 16 : 8;                 // K per instruction
    constexpr int KSTEPS = 64 / (MMA_K * (HALF ? 2 : 4));  // 2
    constexpr uint32_t FMT = PREC == 2 ? 1u : (PREC == 4 ? 0u : 2u);
    constexpr int NACC = 2;                              // accumulator pairs in rotation
    constexpr int BNC = 128;                             // complex columns per tile

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
    __shared__ uint64_t acc_full[NACC], acc_empty[NACC];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ int consumed;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int64_t b = blockIdx.z % a.nbatch;
    const int inst = (int)(blockIdx.z / a.nbatch);
    const int sp = blockIdx.y, nsplit = gridDim.y;
    const InstanceInfo& in = a.in;
    const int64_t slice = a.ctl->slice + (int64_t)inst * in.slice_step;
    if (slice >= a.ctl->slice_end) return;  // idle instance: before any barrier or TMEM
    const TcGeom geo = tc_geom(a, true, PREC);
    const int nkl = (int)(geo.nkb / nsplit);   // k-blocks of this K part
    const int64_t kb0 = (int64_t)sp * nkl;
    const int tiles_m = (int)(geo.rows_r / kBM), tiles_n = (int)(geo.cols_q / BNC);
    int tm, tn;
    {
        const int per_group = kGroupRows * tiles_n;
        const int grp = (int)blockIdx.x / per_group;
        const int first = grp * kGroupRows;
        const int gsz = min(kGroupRows, tiles_m - first);
        const int r = (int)blockIdx.x - grp * per_group;
        tm = first + r % gsz;
        tn = r / gsz;
    }
    const int row0 = tm * kBM, col0 = tn * BNC;
    const char* pk = reinterpret_cast<const char*>(a.P) + (int64_t)inst * in.p_is * 8;

    ScaleIO sio = a.sc;
    if (sio.max_a) sio.max_a += (int64_t)inst * in.sa_is;
    if (sio.exp_a) sio.exp_a += (int64_t)inst * in.sa_is;
    if (sio.max_b) sio.max_b += (int64_t)inst * in.sb_is;
    if (sio.exp_b) sio.exp_b += (int64_t)inst * in.sb_is;
    sio.max_c += (int64_t)inst * in.sc_is;
    sio.exp_c += (int64_t)inst * in.sc_is;
    const int eA = exp_of(sio.max_a), eB = exp_of(sio.max_b);
    const int resid = (eA - max(-120, min(120, eA))) + (eB - max(-120, min(120, eB))) +
                      (PREC == 4 ? 2 * kF16Shift : 0);
    if (blockIdx.x == 0 && sp == 0 && b == 0 && tid == 0 && sio.exp_c)
        *sio.exp_c = (sio.exp_a ? *sio.exp_a : 0) + (sio.exp_b ? *sio.exp_b : 0) + eA + eB;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        for (int q = 0; q < NACC; ++q) {
            mbar_init(&acc_full[q], 1);
            mbar_init(&acc_empty[q], 8);  // one arrival per epilogue warp
        }
        abort_flag = 0;
        consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(512u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ---------------- bulk-copy producer ----------------
        if (tid == 0) {
            const char* r_src = pk + ((b * tiles_m + tm) * geo.nkb + kb0) * PT;
            const char* q_src = pk + geo.region_r + ((b * tiles_n + tn) * geo.nkb + kb0) * PT;
            int issued = 0;
            for (int j = 0; j < nkl; ++j) {
                const int s = j % STAGES;
                if (j >= STAGES &&
                    !mbar_wait(&empty_bar[s], (uint32_t)(((j / STAGES) + 1) & 1), &abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                uint8_t* st = smem + s * STAGE_BYTES;
                mbar_expect_tx(&full_bar[s], STAGE_BYTES);
                const int64_t o = (int64_t)j * PT;
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    bulk_load(st + p * PT, r_src + p * geo.plane_r + o, PT, &full_bar[s]);
                    bulk_load(st + (4 + p) * PT, q_src + p * geo.plane_q + o, PT, &full_bar[s]);
                }
                ++issued;
            }
            if (abort_flag) {
                int dummy = 0;
                for (int j = *(volatile int*)&consumed; j < issued; ++j)
                    mbar_wait(&full_bar[j % STAGES], (uint32_t)((j / STAGES) & 1), &dummy);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (tid == 32) {
            const uint32_t idesc = instr_desc(FMT, kBM, BNC);
            const uint32_t idesc_neg = idesc | (1u << 13);  // negate A: - Im R Im Q
            for (int j = 0; j < nkl; ++j) {
                const int s = j % STAGES;
                if (!mbar_wait(&full_bar[s], (uint32_t)((j / STAGES) & 1), &abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                const int q = j % NACC;
                // an accumulator pair is reused once the epilogue has drained it
                if (j >= NACC && !mbar_wait(&acc_empty[q], (uint32_t)(((j / NACC) + 1) & 1), &abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
                const uint32_t d_re = tmem + (uint32_t)(q * 2 * BNC), d_im = d_re + (uint32_t)BNC;
                // the small hi*lo and lo*hi products first, the large hi*hi ones
                // last (see k_umma: the adder drops bits relative to the larger
                // operand)
#pragma unroll
                for (int k = 0; k < KSTEPS; ++k) {
                    const uint32_t off = k * 32;
                    const uint64_t rrh = smem_desc64(base + 0 * PT + off), rrl = smem_desc64(base + 1 * PT + off);
                    const uint64_t rih = smem_desc64(base + 2 * PT + off), ril = smem_desc64(base + 3 * PT + off);
                    const uint64_t qrh = smem_desc64(base + 4 * PT + off), qrl = smem_desc64(base + 5 * PT + off);
                    const uint64_t qih = smem_desc64(base + 6 * PT + off), qil = smem_desc64(base + 7 * PT + off);
                    const uint32_t acc0 = k > 0 ? 1u : 0u;
                    mma<HALF>(d_re, rrh, qrl, idesc, acc0);
                    mma<HALF>(d_im, rrh, qil, idesc, acc0);
                    mma<HALF>(d_re, rrl, qrh, idesc, 1u);
                    mma<HALF>(d_im, rrl, qih, idesc, 1u);
                    mma<HALF>(d_re, rih, qil, idesc_neg, 1u);
                    mma<HALF>(d_im, rih, qrl, idesc, 1u);
                    mma<HALF>(d_re, ril, qih, idesc_neg, 1u);
                    mma<HALF>(d_im, ril, qrh, idesc, 1u);
                }
#pragma unroll
                for (int k = 0; k < KSTEPS; ++k) {
                    const uint32_t off = k * 32;
                    const uint64_t rrh = smem_desc64(base + 0 * PT + off), rih = smem_desc64(base + 2 * PT + off);
                    const uint64_t qrh = smem_desc64(base + 4 * PT + off), qih = smem_desc64(base + 6 * PT + off);
                    mma<HALF>(d_re, rrh, qrh, idesc, 1u);
                    mma<HALF>(d_im, rrh, qih, idesc, 1u);
                    mma<HALF>(d_re, rih, qih, idesc_neg, 1u);
                    mma<HALF>(d_im, rih, qrh, idesc, 1u);
                }
                mma_commit(&empty_bar[s]);
                mma_commit(&acc_full[q]);
                *(volatile int*)&consumed = j + 1;
            }
            mma_commit(&done_bar);  // arrives once every MMA issued above has completed
        }
    } else {
        // ---------------- epilogue (warps 2..9) ----------------
        float lmax = 0.f;
        const int quad = warp & 3;                 // TMEM lanes 32*quad.. belong to this warp
        const int cbase = ((warp - 2) >> 2) * 64;  // this warp's 64 of the 128 complex columns
        float sre[64], sim[64];
#pragma unroll
        for (int i = 0; i < 64; ++i) {
            sre[i] = 0.f;
            sim[i] = 0.f;
        }
        bool ok = true;
        for (int j = 0; j < nkl && ok; ++j) {
            const int q = j % NACC;
            const bool got = mbar_wait(&acc_full[q], (uint32_t)((j / NACC) & 1), &abort_flag);
            ok = __all_sync(0xffffffffu, got && !abort_flag);  // tcgen05.ld is warp-collective
            if (!ok) break;
            tc_fence_after();
            const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(q * 2 * BNC + cbase);
            tmem_add32(ta, sre);
            tmem_add32(ta + 32u, sre + 32);
            tmem_add32(ta + (uint32_t)BNC, sim);
            tmem_add32(ta + (uint32_t)BNC + 32u, sim + 32);
            tc_fence_before();
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(&acc_empty[q]);
        }
        if (ok) {
            const int row = row0 + quad * 32 + (tid & 31);
            const int64_t M = int64_t(1) << a.nm, N = int64_t(1) << a.nn;
            float* C = nsplit > 1
                           ? reinterpret_cast<float*>(const_cast<char*>(pk) + geo.part_off) +
                                 (int64_t)sp * a.nbatch * M * N * 2
                           : reinterpret_cast<float*>(a.C) + (int64_t)inst * in.c_is * 2;
            const int rs = nsplit > 1 ? 0 : resid;
#pragma unroll
            for (int i = 0; i < 64; ++i) {
                if (rs) {
                    sre[i] = ldexpf(sre[i], -rs);
                    sim[i] = ldexpf(sim[i], -rs);
                }
                lmax = fmaxf(lmax, fmaxf(fabsf(sre[i]), fabsf(sim[i])));
            }
            const int64_t j0 = col0 + cbase;  // first complex column of this warp
            if (!a.tc_swap) {
                float* crow = C + ((b * M + row) * N + j0) * 2;
#pragma unroll
                for (int i = 0; i < 64; i += 2)
                    *reinterpret_cast<float4*>(crow + 2 * i) = make_float4(sre[i], sim[i], sre[i + 1], sim[i + 1]);
            } else {
                // rows run over N, complex columns over M
#pragma unroll
                for (int i = 0; i < 64; ++i)
                    *reinterpret_cast<float2*>(C + ((b * M + j0 + i) * N + row) * 2) = make_float2(sre[i], sim[i]);
            }
        } else if ((tid & 31) == 0) {
            atomicExch(const_cast<int32_t*>(&a.ctl->status), (int32_t)TN_ETIMEOUT);
        }
        if (nsplit == 1) {
            for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
            if ((tid & 31) == 0 && lmax > 0.f) atomicMax(sio.max_c, __float_as_uint(lmax));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        // no MMA may still write the accumulators when they are freed
        int dummy = 0;
        bool quiet = true;
        if (tid == 32) quiet = mbar_wait(&done_bar, 0u, &dummy);
        quiet = __shfl_sync(0xffffffffu, quiet, 0);
        tc_fence_after();
        if (!quiet && tid == 32) atomicExch(const_cast<int32_t*>(&a.ctl->status), (int32_t)TN_ETIMEOUT);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
    }
    if (a.t_done && tid == 0 && nsplit == 1) {
        unsigned long long tnow;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(tnow));
        atomicMax(a.t_done, tnow);
    }
}

// ---------------------------------------------------------------------------
// k_umma3m: complex node as three real TF32 GEMMs (3M) over the Re, Im and
// Re + Im planes of R and Q, one accumulator each (128 complex columns per
// tile); the epilogue forms Re C = T1 - T2 and Im C = T3 - T1 - T2.
// ---------------------------------------------------------------------------
template <int STAGES>
__global__ void __launch_bounds__(kGemmThreads, 1) k_umma3m(const __grid_constant__ TileArgs a) {
    constexpr int STAGE_BYTES = 6 * kTileBytes;
    constexpr int KE = 32, MMA_K = 8, KSTEPS = KE / MMA_K;
    constexpr uint32_t ALLOC = 512;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ int consumed;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int64_t b = blockIdx.z % a.nbatch;
    const int inst = (int)(blockIdx.z / a.nbatch);
    const int sp = blockIdx.y, nsplit = gridDim.y;
    const InstanceInfo& in = a.in;
    const int64_t slice = a.ctl->slice + (int64_t)inst * in.slice_step;
    if (slice >= a.ctl->slice_end) return;
    const TcGeom geo = tc_geom(a, true, 3);
    const int nkl = (int)(geo.nkb / nsplit);
    const int64_t kb0 = (int64_t)sp * nkl;
    const int tiles_m = (int)(geo.rows_r / kBM), tiles_n = (int)(geo.cols_q / kBN);
    int tm, tn;
    {
        const int per_group = kGroupRows * tiles_n;
        const int grp = (int)blockIdx.x / per_group;
        const int first = grp * kGroupRows;
        const int gsz = min(kGroupRows, tiles_m - first);
        const int r = (int)blockIdx.x - grp * per_group;
        tm = first + r % gsz;
        tn = r / gsz;
    }
    const int row0 = tm * kBM, col0 = tn * kBN;
    const char* pk = reinterpret_cast<const char*>(a.P) + (int64_t)inst * in.p_is * 8;
    ScaleIO sio = a.sc;
    if (sio.max_a) sio.max_a += (int64_t)inst * in.sa_is;
    if (sio.exp_a) sio.exp_a += (int64_t)inst * in.sa_is;
    if (sio.max_b) sio.max_b += (int64_t)inst * in.sb_is;
    if (sio.exp_b) sio.exp_b += (int64_t)inst * in.sb_is;
    sio.max_c += (int64_t)inst * in.sc_is;
    sio.exp_c += (int64_t)inst * in.sc_is;
    const int eA = exp_of(sio.max_a), eB = exp_of(sio.max_b);
    const int resid = (eA - max(-120, min(120, eA))) + (eB - max(-120, min(120, eB)));
    if (blockIdx.x == 0 && sp == 0 && b == 0 && tid == 0 && sio.exp_c)
        *sio.exp_c = (sio.exp_a ? *sio.exp_a : 0) + (sio.exp_b ? *sio.exp_b : 0) + eA + eB;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(ALLOC));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (tid == 0) {
            const char* r_src = pk + ((b * tiles_m + tm) * geo.nkb + kb0) * kTileBytes;
            const char* q_src = pk + geo.region_r + ((b * tiles_n + tn) * geo.nkb + kb0) * kTileBytes;
            int issued = 0;
            for (int j = 0; j < nkl; ++j) {
                const int s = j % STAGES;
                if (j >= STAGES &&
                    !mbar_wait(&empty_bar[s], (uint32_t)(((j / STAGES) + 1) & 1), &abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                uint8_t* st = smem + s * STAGE_BYTES;
                mbar_expect_tx(&full_bar[s], STAGE_BYTES);
                const int64_t o = (int64_t)j * kTileBytes;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    bulk_load(st + q * kTileBytes, r_src + q * geo.plane_r + o, kTileBytes, &full_bar[s]);
                    bulk_load(st + (3 + q) * kTileBytes, q_src + q * geo.plane_q + o, kTileBytes, &full_bar[s]);
                }
                ++issued;
            }
            if (abort_flag) {
                int dummy = 0;
                for (int j = *(volatile int*)&consumed; j < issued; ++j)
                    mbar_wait(&full_bar[j % STAGES], (uint32_t)((j / STAGES) & 1), &dummy);
            }
        }
    } else if (warp == 1) {
        if (tid == 32) {
            const uint32_t idesc = instr_desc(2u, kBM, kBN);
            for (int j = 0; j < nkl; ++j) {
                const int s = j % STAGES;
                if (!mbar_wait(&full_bar[s], (uint32_t)((j / STAGES) & 1), &abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
                for (int k = 0; k < KSTEPS; ++k) {
                    const uint32_t off = k * MMA_K * 4;
                    const uint32_t acc = (j > 0 || k > 0) ? 1u : 0u;
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        mma<false>(tmem + (uint32_t)(q * kBN), smem_desc(base + q * kTileBytes + off),
                                   smem_desc(base + (3 + q) * kTileBytes + off), idesc, acc);
                }
                mma_commit(&empty_bar[s]);
                *(volatile int*)&consumed = j + 1;
            }
            mma_commit(&done_bar);
        }
    } else {
        float lmax = 0.f;
        const bool done0 = mbar_wait(&done_bar, 0u, &abort_flag);
        tc_fence_after();
        const bool done = __all_sync(0xffffffffu, done0 && !abort_flag);
        if (done) {
            const int quad = warp & 3;
            const int row = row0 + quad * 32 + (tid & 31);
            const int64_t M = int64_t(1) << a.nm, N = int64_t(1) << a.nn;
            float* C = nsplit > 1
                           ? reinterpret_cast<float*>(const_cast<char*>(pk) + geo.part_off) +
                                 (int64_t)sp * a.nbatch * M * N * 2
                           : reinterpret_cast<float*>(a.C) + (int64_t)inst * in.c_is * 2;
            const int rs = nsplit > 1 ? 0 : resid;
            for (int col = 0; col < kBN; col += 16) {
                float t1[16], t2[16], t3[16];
                const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)col;
                tmem_ld16(ta, t1);
                tmem_ld16(ta + kBN, t2);
                tmem_ld16(ta + 2 * kBN, t3);
                float re[16], im[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    re[i] = t1[i] - t2[i];
                    im[i] = t3[i] - t1[i] - t2[i];
                    if (rs) {
                        re[i] = ldexpf(re[i], -rs);
                        im[i] = ldexpf(im[i], -rs);
                    }
                    lmax = fmaxf(lmax, fmaxf(fabsf(re[i]), fabsf(im[i])));
                }
                const int64_t j0 = col0 + col;  // first complex column of the chunk
                if (!a.tc_swap) {
                    float* crow = C + ((b * M + row) * N + j0) * 2;
#pragma unroll
                    for (int i = 0; i < 16; i += 2)
                        *reinterpret_cast<float4*>(crow + 2 * i) = make_float4(re[i], im[i], re[i + 1], im[i + 1]);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        *reinterpret_cast<float2*>(C + ((b * M + j0 + i) * N + row) * 2) = make_float2(re[i], im[i]);
                }
            }
        } else if ((tid & 31) == 0) {
            atomicExch(const_cast<int32_t*>(&a.ctl->status), (int32_t)TN_ETIMEOUT);
        }
        if (nsplit == 1) {
            for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
            if ((tid & 31) == 0 && lmax > 0.f) atomicMax(sio.max_c, __float_as_uint(lmax));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        int dummy = 0;
        bool quiet = true;
        if (tid == 32) quiet = mbar_wait(&done_bar, 0u, &dummy);
        quiet = __shfl_sync(0xffffffffu, quiet, 0);
        tc_fence_after();
        if (!quiet && tid == 32) atomicExch(const_cast<int32_t*>(&a.ctl->status), (int32_t)TN_ETIMEOUT);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ALLOC));
    }
    if (a.t_done && tid == 0 && nsplit == 1) {
        unsigned long long tnow;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(tnow));
        atomicMax(a.t_done, tnow);
    }
}

// ---------------------------------------------------------------------------
// k_tc_reduce: C = sum of the K parts in part order (FP32), the residual
// renormalisation and the node maximum.  blockIdx.y: instance.
// ---------------------------------------------------------------------------
template <bool CPLX, int PREC>
__global__ void __launch_bounds__(256) k_tc_reduce(const __grid_constant__ TileArgs a) {
    const int inst = blockIdx.y;
    const InstanceInfo& in = a.in;
    const int64_t slice = a.ctl->slice + (int64_t)inst * in.slice_step;
    if (slice >= a.ctl->slice_end) return;
    const TcGeom geo = tc_geom(a, CPLX, PREC);
    const int ESZ = CPLX ? 8 : 4;
    const int64_t n4 = (a.nbatch << (a.nm + a.nn)) * (CPLX ? 2 : 1) / 4;  // float4 per part
    const float4* P = reinterpret_cast<const float4*>(reinterpret_cast<const char*>(a.P) +
                                                      (int64_t)inst * in.p_is * ESZ + geo.part_off);
    float4* C = reinterpret_cast<float4*>(reinterpret_cast<float*>(a.C) + (int64_t)inst * in.c_is * (CPLX ? 2 : 1));
    ScaleIO sio = a.sc;
    if (sio.max_a) sio.max_a += (int64_t)inst * in.sa_is;
    if (sio.max_b) sio.max_b += (int64_t)inst * in.sb_is;
    sio.max_c += (int64_t)inst * in.sc_is;
    const int eA = exp_of(sio.max_a), eB = exp_of(sio.max_b);
    const int resid = (eA - max(-120, min(120, eA))) + (eB - max(-120, min(120, eB))) +
                      (PREC == 4 ? 2 * kF16Shift : 0);
    float lmax = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        float4 s = P[i];
        for (int p = 1; p < a.split; ++p) {
            const float4 t = P[p * n4 + i];
            s.x += t.x; s.y += t.y; s.z += t.z; s.w += t.w;
        }
        if (resid) {
            s.x = ldexpf(s.x, -resid); s.y = ldexpf(s.y, -resid);
            s.z = ldexpf(s.z, -resid); s.w = ldexpf(s.w, -resid);
        }
        lmax = fmaxf(lmax, fmaxf(fmaxf(fabsf(s.x), fabsf(s.y)), fmaxf(fabsf(s.z), fabsf(s.w))));
        C[i] = s;
    }
    for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if ((threadIdx.x & 31) == 0 && lmax > 0.f) atomicMax(sio.max_c, __float_as_uint(lmax));
    if (a.t_done && threadIdx.x == 0) {
        unsigned long long tnow;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(tnow));
        atomicMax(a.t_done, tnow);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

// Host copies of the tile layouts (swz, swz64 above).
inline int64_t host_swz128(int64_t row, int64_t chunk) {
    return (row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4);
}
inline int64_t host_swz64(int64_t row, int64_t chunk) {
    return (row >> 3) * 512 + (row & 7) * 64 + ((chunk ^ ((row >> 1) & 3)) << 4);
}

// Byte position in the first packed plane of operand entry (row, k) (row
// counts batch entries x rows, k the complex or real K index), for the
// layout the kernels read: planar, 3M, 4M (R interleaves (re, im) along K,
// Q's column c becomes rows 2c and 2c + 1) or real.
int64_t packed_pos(const TcGeom& g, int prec, bool cplx, int role, int64_t row, int64_t k) {
    const int lg_esz = g.esz == 2 ? 1 : 2;
    if (g.planar) {
        const int lg_ke = 6 - lg_esz;
        const int64_t tile = (row >> 7) * g.nkb + (k >> lg_ke);
        const int64_t byte = (k & ((int64_t(1) << lg_ke) - 1)) << lg_esz;
        return tile * (kTileBytes / 2) + host_swz64(row & 127, byte >> 4) + (byte & 15);
    }
    int64_t rr = row, kk = k;
    if (cplx && prec != 3) {
        kk = 2 * k;
        if (role == 1) rr = 2 * row;
    }
    const int lg_ke = 7 - lg_esz;
    const int64_t tile = (rr >> 7) * g.nkb + (kk >> lg_ke);
    const int64_t byte = (kk & ((int64_t(1) << lg_ke) - 1)) << lg_esz;
    return tile * kTileBytes + host_swz128(rr & 127, byte >> 4) + (byte & 15);
}

// Tile bits of a pack (role 0: R, 1: Q): the kPackLow lowest packed
// positions and the kPackLow lowest source strides, filled up with the next
// packed positions to 2 * kPackLow bits; the other bits enumerate tiles.
// Destination byte positions: one XOR constant per packed-index bit.
PackPlan make_pack_plan(const TileArgs& a, int role, int prec, bool cplx) {
    PackPlan pp;
    memset(&pp, 0, sizeof(pp));
    const bool useB = (role == 0) == (a.tc_swap != 0);
    const int nk = a.nk, no = useB ? a.nn : a.nm, nb = a.nb;
    const int nbits = nk + no + nb;
    const TcGeom geo = tc_geom(a, cplx, prec);
    int64_t lpos[3 * kMaxBits];
    for (int p = 0; p < nbits; ++p) {
        // Q's batch entries start on whole (padded) 128-row tiles
        const int pad = role == 1 && p >= nk + no ? geo.q_pad_lg : 0;
        const int64_t row = p >= nk ? int64_t(1) << (p - nk + pad) : 0;
        const int64_t k = p < nk ? int64_t(1) << p : 0;
        lpos[p] = packed_pos(geo, prec, cplx, role, row, k);
    }
    pp.pos_row1 = host_swz128(1, 0);  // row 2c + 1 of the 4M layout from row 2c
    const uint8_t* xk = useB ? a.b_k : a.a_k;
    const uint8_t* xo = useB ? a.b_n : a.a_m;
    const uint8_t* xb = useB ? a.b_b : a.a_b;
    uint8_t shift[3 * kMaxBits];
    for (int p = 0; p < nbits; ++p) shift[p] = p < nk ? xk[p] : (p < nk + no ? xo[p - nk] : xb[p - nk - no]);
    int by_shift[64];
    for (int s = 0; s < 64; ++s) by_shift[s] = -1;
    for (int p = 0; p < nbits; ++p)
        if (shift[p] < 64) by_shift[shift[p]] = p;  // kNoBit: a K bit the operand lacks
    bool in_tile[3 * kMaxBits];
    for (int p = 0; p < nbits; ++p) in_tile[p] = p < kPackLow;
    for (int s = 0, r = 0; s < 64 && r < kPackLow; ++s)
        if (by_shift[s] >= 0) {
            in_tile[by_shift[s]] = true;
            ++r;
        }
    int cnt = 0;
    for (int p = 0; p < nbits; ++p) cnt += in_tile[p];
    for (int p = kPackLow; p < nbits && cnt < 2 * kPackLow; ++p)
        if (!in_tile[p]) {
            in_tile[p] = true;
            ++cnt;
        }
    int td[2 * kPackLow], ts[2 * kPackLow];
    int t = 0, u = 0;
    for (int p = 0; p < nbits; ++p) {
        if (in_tile[p]) {
            td[t++] = p;
        } else {
            pp.rest_src[u] = shift[p] < 64 ? int64_t(1) << shift[p] : 0;
            pp.rest_pos[u] = lpos[p];
            ++u;
        }
    }
    // the same tile bits in source order (ascending stride; absent bits,
    // which repeat the same source value, last)
    int w = 0;
    for (int s = 0; s < 64; ++s)
        if (by_shift[s] >= 0 && in_tile[by_shift[s]]) ts[w++] = by_shift[s];
    for (int i = 0; i < t; ++i)
        if (shift[td[i]] >= 64) ts[w++] = td[i];
    for (int j = 0; j < t; ++j) {
        pp.src_add[j] = shift[ts[j]] < 64 ? int64_t(1) << shift[ts[j]] : 0;
        pp.dst_pos[j] = lpos[td[j]];
        int r = 0;
        while (ts[r] != td[j]) ++r;
        pp.idx_add[j] = 1 << r;
    }
    pp.t = t;
    pp.u = u;
    return pp;
}

cudaError_t launch_tc_3m(const TileArgs& a, cudaStream_t s) {
    constexpr int STAGES = 2;
    constexpr int SMEM = STAGES * 6 * kTileBytes + 1024;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_umma3m<STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const TcGeom g = tc_geom(a, true, 3);
    const int ni = a.in.n_inst > 1 ? a.in.n_inst : 1;
    const int split = a.split > 1 ? a.split : 1;
    if (g.nkb % split) return cudaErrorInvalidValue;
    const int64_t elems_a = int64_t(1) << (a.nk + a.nm + a.nb);
    const int64_t elems_b = int64_t(1) << (a.nk + a.nn + a.nb);
    auto blocks = [ni](int64_t n) { return pack_blocks(n, ni); };
    if (g.kr < g.ke) {
        // K shorter than one packed row: the rest of every row must be zero
        const size_t pitch = (size_t)(a.in.n_inst > 1 ? a.in.p_is * 8 : g.part_off);
        cudaError_t e0 = cudaMemset2DAsync(a.P, pitch, 0, (size_t)g.part_off, (size_t)ni, s);
        if (e0 != cudaSuccess) return e0;
    }
    {
        const unsigned br = blocks(a.tc_swap ? elems_b : elems_a), bq = blocks(a.tc_swap ? elems_a : elems_b);
        k_pack<true, 3><<<dim3(br + bq, ni), kPackThreads, 0, s>>>(a, make_pack_plan(a, 0, 3, true),
                                                                 make_pack_plan(a, 1, 3, true), (int)br);
    }
    const int64_t tiles = (g.rows_r / kBM) * (g.cols_q / kBN);
    k_umma3m<STAGES><<<dim3((unsigned)tiles, (unsigned)split, (unsigned)(a.nbatch * ni)), kGemmThreads, SMEM, s>>>(a);
    if (split > 1) {
        const int64_t n4 = (a.nbatch << (a.nm + a.nn)) * 2 / 4;
        const unsigned nb = (unsigned)std::min<int64_t>(std::max<int64_t>((n4 + 255) / 256, 1), (int64_t)sm_count() * 8);
        k_tc_reduce<true, 3><<<dim3(nb, ni), 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// Row tiles per raster group of the persistent GEMMs: the group's packed R
// rows (all of K) stay in L2 while the column tiles stream past them, so the
// group holds at most a quarter of L2 of them (at least one row tile, two
// for CTA pairs, at most 32).
int group_rows(const TileArgs& a, bool cplx, int prec, bool pair) {
    static int l2 = 0;
    if (!l2) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev) == cudaSuccess &&
            v > 0)
            l2 = v;
        else
            l2 = 126 << 20;
        cudaGetLastError();
    }
    const TcGeom g = tc_geom(a, cplx, prec);
    const int nsplit = a.split > 1 ? a.split : 1;
    const int64_t row_bytes = std::max<int64_t>(g.nkb / nsplit, 1) * kTileBytes * g.parts;
    int64_t rows = (int64_t)(l2 / 4) / row_bytes;
    rows = std::max<int64_t>(std::min<int64_t>(rows, kGroupRows), pair ? 2 : 1);
    if (pair) rows &= ~int64_t(1);
    return (int)rows;
}

// pipeline depth: as many stages as fit in 192 KB
template <int PREC, int BN>
constexpr int stages_of() {
    return (192 * 1024) / ((PREC == 0 ? 1 : 2) * (kTileBytes + BN * kRowBytes));
}

template <bool CPLX, int PREC, int BN>
cudaError_t launch_umma(const TileArgs& a, dim3 grid, int nacc, cudaStream_t s) {
    constexpr int STAGES = stages_of<PREC, BN>();
    constexpr int SMEM = STAGES * (PREC == 0 ? 1 : 2) * (kTileBytes + BN * kRowBytes) + 1024;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_umma<CPLX, PREC, STAGES, BN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    // persistent: at most one CTA per SM (the stages fill its shared memory),
    // each walking every gridDim.x-th work item
    const int64_t items = (int64_t)grid.x * grid.y * grid.z;
    const unsigned ctas = (unsigned)std::min<int64_t>(items, (int64_t)sm_count());
    k_umma<CPLX, PREC, STAGES, BN><<<ctas, 64 + BN, SMEM, s>>>(a, nacc, group_rows(a, CPLX, PREC, false));
    return cudaGetLastError();
}

// CTA pairs: 64 KB stages (split precisions), as many as fit in 192 KB;
// persistent over the pair items, at most as many pairs as fit at once
template <bool CPLX, int PREC, int BN>
cudaError_t launch_umma2(const TileArgs& a, int64_t items, int nacc, cudaStream_t s) {
    constexpr int STAGE_BYTES = (PREC == 0 ? 1 : 2) * (kTileBytes + BN / 2 * kRowBytes);
    constexpr int STAGES = (192 * 1024) / STAGE_BYTES;
    constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
    auto* kern = k_umma2<CPLX, PREC, STAGES, BN>;
    static bool configured = false;
    static int max_pairs = 0;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(320);
    cfg.dynamicSmemBytes = SMEM;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        cfg.gridDim = dim3((unsigned)(sm_count() & ~1));
        e = cudaOccupancyMaxActiveClusters(&max_pairs, kern, &cfg);
        if (e != cudaSuccess) return e;
        if (max_pairs < 1) return cudaErrorInvalidConfiguration;
        configured = true;
    }
    const unsigned pairs = (unsigned)std::min<int64_t>(items / 2, (int64_t)max_pairs);
    cfg.gridDim = dim3(2 * pairs);
    cfg.stream = s;
    return cudaLaunchKernelEx(&cfg, kern, a, nacc, group_rows(a, CPLX, PREC, true));
}

// planar layout: 64 KB stages, three in flight
template <int PREC>
cudaError_t launch_umma_planar(const TileArgs& a, dim3 grid, cudaStream_t s) {
    constexpr int STAGES = 3;
    constexpr int SMEM = STAGES * 8 * (kTileBytes / 2) + 1024;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_umma_planar<PREC, STAGES>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_umma_planar<PREC, STAGES><<<grid, 320, SMEM, s>>>(a);
    return cudaGetLastError();
}

template <bool CPLX, int PREC>
cudaError_t launch_tc_t(const TileArgs& a, cudaStream_t s) {
    const TcGeom g = tc_geom(a, CPLX, PREC);
    const int ni = a.in.n_inst > 1 ? a.in.n_inst : 1;
    const int split = a.split > 1 ? a.split : 1;
    if (g.nkb % split) return cudaErrorInvalidValue;
    const int64_t elems_a = int64_t(1) << (a.nk + a.nm + a.nb);
    const int64_t elems_b = int64_t(1) << (a.nk + a.nn + a.nb);
    auto blocks = [ni](int64_t n) { return pack_blocks(n, ni); };
    const int64_t n_r = a.tc_swap ? elems_b : elems_a, n_q = a.tc_swap ? elems_a : elems_b;
    if (g.kr < g.ke) {
        // K shorter than one packed row: the rest of every row must be zero
        const size_t pitch = (size_t)(a.in.n_inst > 1 ? a.in.p_is * (CPLX ? 8 : 4) : g.part_off);
        cudaError_t e0 = cudaMemset2DAsync(a.P, pitch, 0, (size_t)g.part_off, (size_t)ni, s);
        if (e0 != cudaSuccess) return e0;
    }
    // pack grid: both operands' blocks in at most one round of resident CTAs
    // (per instance), shared in proportion to the bytes each operand moves,
    // so that no second, partly filled round of blocks trails the launch
    unsigned br = blocks(n_r), bq = blocks(n_q);
    {
        static int per_sm = 0;
        if (!per_sm) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pack<CPLX, PREC>, kPackThreads, 0) !=
                    cudaSuccess ||
                per_sm < 1)
                per_sm = 1;
            cudaGetLastError();
        }
        const int64_t slots = std::max<int64_t>((int64_t)per_sm * sm_count() / ni, 2);
        if ((int64_t)br + bq > slots) {
            const int src = CPLX ? 8 : 4;
            const double wr = (double)n_r * (src + g.parts * g.esz * (CPLX ? 2 : 1));
            const double wq = (double)n_q * (src + g.parts * g.esz * (CPLX ? (g.planar ? 2 : 4) : 1));
            int64_t r = (int64_t)std::llround((double)slots * wr / (wr + wq));
            r = std::min<int64_t>(std::max<int64_t>(r, 1), slots - 1);
            br = (unsigned)std::min<int64_t>(r, br);
            bq = (unsigned)std::min<int64_t>(slots - r, bq);
        }
    }
    k_pack<CPLX, PREC><<<dim3(br + bq, ni), kPackThreads, 0, s>>>(a, make_pack_plan(a, 0, PREC, CPLX),
                                                                 make_pack_plan(a, 1, PREC, CPLX), (int)br);
    const int nkl = (int)(g.nkb / split);
    const int chains = (nkl + umma_chain(PREC) - 1) / umma_chain(PREC);
    const int max_acc = 512 / g.bn;
    const int nacc = chains >= max_acc ? max_acc : (chains >= 2 ? 2 : 1);
    const int64_t tiles = (g.rows_r / kBM) * (g.cols_q / g.bn);
    dim3 grid((unsigned)tiles, (unsigned)split, (unsigned)(a.nbatch * ni));
    // 256-column tiles over an even number of row tiles run on CTA pairs
    const bool pair = g.bn == 256 && !g.planar && (g.rows_r / kBM) % 2 == 0 && !a.tc_nopair;
    // padded (narrow) column operands: only k_umma keeps the valid columns
    if (g.cols_valid != g.cols_q && (g.planar || pair || g.bn != kBN)) return cudaErrorInvalidValue;
    cudaError_t e;
    if constexpr (CPLX && (PREC == 1 || PREC == 2 || PREC == 4)) {
        if (g.planar) {
            e = launch_umma_planar<PREC>(a, grid, s);
        } else if (pair) {
            e = launch_umma2<CPLX, PREC, 256>(a, (int64_t)grid.x * grid.y * grid.z, nacc, s);
        } else {
            e = g.bn == 256 ? launch_umma<CPLX, PREC, 256>(a, grid, nacc, s)
                            : launch_umma<CPLX, PREC, 128>(a, grid, nacc, s);
        }
    } else if (pair) {
        e = launch_umma2<CPLX, PREC, 256>(a, (int64_t)grid.x * grid.y * grid.z, nacc, s);
    } else {
        e = g.bn == 256 ? launch_umma<CPLX, PREC, 256>(a, grid, nacc, s)
                        : launch_umma<CPLX, PREC, 128>(a, grid, nacc, s);
    }
    if (e != cudaSuccess) return e;
    if (split > 1) {
        const int64_t n4 = (a.nbatch << (a.nm + a.nn)) * (CPLX ? 2 : 1) / 4;
        const unsigned nb = (unsigned)std::min<int64_t>(std::max<int64_t>((n4 + 255) / 256, 1), (int64_t)sm_count() * 8);
        k_tc_reduce<CPLX, PREC><<<dim3(nb, ni), 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc(const TileArgs& a, int prec, bool is_c, cudaStream_t s) {
    prec = tc_prec_of_node(a, is_c, prec);
    if (prec == 3) return launch_tc_3m(a, s);
    if (is_c) {
        if (prec == 0) return launch_tc_t<true, 0>(a, s);
        if (prec == 1) return launch_tc_t<true, 1>(a, s);
        if (prec == 4) return launch_tc_t<true, 4>(a, s);
        return launch_tc_t<true, 2>(a, s);
    }
    if (prec == 0) return launch_tc_t<false, 0>(a, s);
    if (prec == 1) return launch_tc_t<false, 1>(a, s);
    if (prec == 4) return launch_tc_t<false, 4>(a, s);
    return launch_tc_t<false, 2>(a, s);
}

}  // namespace tn
