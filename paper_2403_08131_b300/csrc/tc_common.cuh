// Shared tcgen05 / TMA / mbarrier helpers of the tensor-core kernels (inline PTX, sm_100a+).
#pragma once

#include "gpbo_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

namespace gpbo {
namespace tcx {

constexpr long long TIMEOUT_CYCLES = WAIT_DEFAULT_CYCLES;  // bounded waits: about 2 s of SM clock

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// A wait that honours the abort flag gives up after the context's wait limit (wait_limit).
// The waits with which a CTA drains its own copies and MMAs before it exits always allow
// TIMEOUT_CYCLES, so that a short limit never releases shared or tensor memory that an
// asynchronous operation still uses.

// Failure injection word (byte 4 of the status buffer, gpbo_inject_wait_stall): bit 0 makes the
// tensor-core variance kernel's epilogue wait on a barrier that nothing arrives at.
__device__ __forceinline__ unsigned injected_faults(const unsigned *status)
{
    return *(const volatile unsigned *)(status + 1);
}

// Bounded wait.  Gives up (returning false) when another role has aborted, or after the wait
// limit, in which case it raises the abort flag and the device status bit.
static __device__ __noinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, unsigned *status,
                                       bool honour_abort = true)
{
    long long t0 = clock64();
    const long long limit = honour_abort ? wait_limit(status) : TIMEOUT_CYCLES;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 255u) {
            if (honour_abort && *abort_flag) return false;
            if (clock64() - t0 > limit) {
                *abort_flag = 1;
                atomicOr(status, DEV_TIMEOUT);
                return false;
            }
        }
    }
}

// The same bounded loop, inlined: for hot loops whose waits often miss the first attempt,
// where a call would save and restore live registers through local memory.
__device__ __forceinline__ bool mbar_wait_inl(uint64_t *bar, uint32_t parity, volatile int *abort_flag, unsigned *status)
{
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 0u) {
            if (*abort_flag) return false;
            if (clock64() - t0 > wait_limit(status)) {
                *abort_flag = 1;
                atomicOr(status, DEV_TIMEOUT);
                return false;
            }
        }
    }
}

// The same wait with its first attempt inline: the out-of-line slow path (and the register
// saves around its call) only runs when the barrier is not ready at once.
__device__ __forceinline__ bool mbar_wait_fast(uint64_t *bar, uint32_t parity, volatile int *abort_flag, unsigned *status,
                                               bool honour_abort = true)
{
    if (mbar_try(bar, parity)) return true;
    return mbar_wait(bar, parity, abort_flag, status, honour_abort);
}

// The same, multicast: the box lands at dst's offset in every CTA of `mask` (this GPU's own
// memory only), and each of them counts its bytes on the mbarrier at bar's offset.
__device__ __forceinline__ void tma_load_2d_mc(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar,
                                               uint16_t mask)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1, {%2, "
        "%3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar)), "h"(mask)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Error-free 8-bit slicing on the integer pipe (no FP64 instruction).  For x with |x| < 2^e,
// fixed_of(x, e, P) returns X = round(x 2^(P - e)) (|X| <= 2^P) from the bits of x, and
// split_digits<S> writes X = sum_s d_s 2^(8 (S - 1 - s)) in balanced base-256 digits, d_0 ..
// d_(S-1) with |d_0| <= 128 (for P = 8 S - 1) and -128 <= d_s <= 127 for s > 0, each as BF16 bits
// (exact: at most 8 significant bits).  |x - X 2^(e - P)| <= 2^(e - P - 1).
__device__ __forceinline__ int64_t fixed_of(double x, int e, int P)
{
    const uint64_t bits = (uint64_t)__double_as_longlong(x), mag = bits & 0x7fffffffffffffffull;
    const int E = (int)(mag >> 52);
    const uint64_t m = (mag & 0x000fffffffffffffull) | (E ? 0x0010000000000000ull : 0ull);
    const int sh = (E ? E : 1) - 1075 + P - e;  // x = m 2^(E - 1075); |x| < 2^e makes X < 2^P
    uint64_t X;
    if (sh >= 0) X = m << sh;
    else if (sh > -64) X = (m + (1ull << (-sh - 1))) >> (-sh);
    else X = 0;
    return (bits >> 63) ? -(int64_t)X : (int64_t)X;
}
__device__ __forceinline__ int64_t fixed_of(float x, int e, int P)
{
    const uint32_t bits = __float_as_uint(x), mag = bits & 0x7fffffffu;
    const int E = (int)(mag >> 23);
    const uint64_t m = (uint64_t)((mag & 0x007fffffu) | (E ? 0x00800000u : 0u));
    const int sh = (E ? E : 1) - 150 + P - e;  // x = m 2^(E - 150)
    uint64_t X;
    if (sh >= 0) X = m << sh;
    else if (sh > -64) X = (m + (1ull << (-sh - 1))) >> (-sh);
    else X = 0;
    return (bits >> 31) ? -(int64_t)X : (int64_t)X;
}
__device__ __forceinline__ int64_t fixed55(double x, int e) { return fixed_of(x, e, 55); }
// |x| as an unsigned integer that orders like |x|
__device__ __forceinline__ uint64_t mag_bits(double x)
{
    return (uint64_t)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ uint64_t mag_bits(float x) { return __float_as_uint(x) & 0x7fffffffu; }
// the exponent e with |x| < 2^e for the largest magnitude mx (as mag_bits), 0 for mx = 0
__device__ __forceinline__ int exp_of_mag(uint64_t mx) { return mx ? (int)(mx >> 52 ? mx >> 52 : 1) - 1022 : 0; }
template <typename T> __device__ __forceinline__ int exp_of_mag_t(uint64_t mx);
template <> __device__ __forceinline__ int exp_of_mag_t<double>(uint64_t mx) { return exp_of_mag(mx); }
template <> __device__ __forceinline__ int exp_of_mag_t<float>(uint64_t mx)
{
    return mx ? (int)(mx >> 23 ? mx >> 23 : 1) - 126 : 0;
}
__device__ __forceinline__ uint16_t bf16_of_small_int(int d)
{
    return (uint16_t)(__float_as_uint((float)d) >> 16);  // |d| <= 128: exact in BF16
}
template <int S> __device__ __forceinline__ void split_digits(int64_t X, uint16_t (&out)[S])
{
#pragma unroll
    for (int s = S - 1; s >= 1; --s) {
        const int64_t q = (X + 128) >> 8;
        out[s] = bf16_of_small_int((int)(X - (q << 8)));
        X = q;
    }
    out[0] = bf16_of_small_int((int)X);
}
__device__ __forceinline__ void split7(int64_t X, uint16_t (&out)[7]) { split_digits<7>(X, out); }

// TMA tile store (shared -> global) in the calling thread's bulk async-group.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"((uint64_t)map),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the group's stores have read their shared-memory source
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// the group's stores are complete
__device__ __forceinline__ void bulk_wait_all0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Shared-memory matrix descriptor for a K-major tile written by TMA with 128-byte
// swizzle: rows of 128 bytes, 8-row atoms 1024 bytes apart (stride byte offset).
__device__ __forceinline__ uint64_t smem_desc(const void *p)
{
    const uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr & 0x3FFFFull) >> 4;          // start address
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                 // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
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


// TMEM loads without the wait, so that several can be in flight; tmem_wait() waits for all
// of them, and pin() then ties the destination registers to that point: an empty volatile asm
// that "modifies" them keeps the compiler from reading them before the wait.
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void pin16(uint32_t *r)
{
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]));
}

// x 2^k as a double, built on the integer pipe: normalise |x| by its leading zeros, write the
// exponent with k folded in and the top 52 bits after the leading one (truncated: relative
// error below 2^-52).  Values outside the normal range take scalbn.  For the FP64 results of
// the slice-product kernels, where the FP64 pipe is the scarce one.
__device__ __forceinline__ double scaled_to_double(long long x, int k)
{
    if (x == 0) return 0.0;
    const unsigned long long sign = (unsigned long long)x & 0x8000000000000000ull;
    const unsigned long long ux = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
    const int lz = __clzll((long long)ux);
    const int ex = 1023 + 63 - lz + k;
    if (ex <= 0 || ex >= 2047) return scalbn((double)x, k);
    const unsigned long long m = (ux << lz) >> 11;
    return __longlong_as_double((long long)(sign | ((unsigned long long)ex << 52) | (m & 0x000FFFFFFFFFFFFFull)));
}

// ---- CTA pairs (clusters of two CTAs whose tensor cores run one MMA together, cta_group::2)
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Every thread of every CTA of the cluster arrives, then waits for all the others.
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared::cluster address of the variable at local shared address p in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(const void *p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}
// Arrive (release, cluster scope) on an mbarrier given by its shared::cluster address.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t caddr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}
// Relaxed arrive (no release fence) on an mbarrier given by its shared::cluster address: for a
// signal that publishes no memory writes of the arriving thread (a stage whose copies another
// barrier has already seen land).
__device__ __forceinline__ void mbar_arrive_cluster_relaxed(uint32_t caddr)
{
    asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}
// try_wait with cluster-scope acquire, for barriers that the peer CTA arrives on.
__device__ __forceinline__ bool mbar_try_cluster(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
static __device__ __noinline__ bool mbar_wait_cluster(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                                      unsigned *status)
{
    const long long t0 = clock64(), limit = wait_limit(status);
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_cluster(bar, parity)) return true;
        if ((it & 255u) == 255u) {
            if (*abort_flag) return false;
            if (clock64() - t0 > limit) {
                *abort_flag = 1;
                atomicOr(status, DEV_TIMEOUT);
                return false;
            }
        }
    }
}
// One MMA of the CTA pair, issued by one thread of the pair's first CTA: D (128 lanes of each
// CTA's tensor memory) += A (each CTA's own 128 rows) x B (N rows: the first half from this
// CTA's shared memory, the second from the peer's, at the same offsets).
__device__ __forceinline__ void mma_f16_pair(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}
// Arrive on the mbarrier at this offset in each CTA of `mask` once the pair's MMAs issued so far
// by this thread are complete.
__device__ __forceinline__ void mma_commit_pair(uint64_t *bar, uint16_t mask)
{
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "h"(mask)
                 : "memory");
}

// Arrive on the mbarrier at this offset in each CTA of `mask` once the (one-CTA) MMAs issued so
// far by this thread are complete.
__device__ __forceinline__ void mma_commit_mc(uint64_t *bar, uint16_t mask)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "h"(mask)
                 : "memory");
}

// Instruction descriptor, kind::f16: FP32 accumulate, A/B format (0 = F16, 1 = BF16), both
// K-major, N x M.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t fmt, int N, int M)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }


}  // namespace tcx

// 2-D row-major 16-bit matrix (rows x cols, cols contiguous), box = box_rows x 64 cols, 128B swizzle.
int encode_2d(CUtensorMap *map, CUtensorMapDataType dt, const void *base, uint64_t rows, uint64_t cols,
              uint32_t box_rows);
// The same with box = box_rows x box_cols and the given swizzle (box_cols x 2 bytes = the swizzle span).
int encode_2d_box(CUtensorMap *map, CUtensorMapDataType dt, const void *base, uint64_t rows, uint64_t cols,
                  uint32_t box_rows, uint32_t box_cols, CUtensorMapSwizzle swizzle);

}  // namespace gpbo
