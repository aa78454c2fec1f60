// matmul_tc.cu -- the tensor-core path of the secret-shared matrix product
// (Sec. III-D.3 product Z_i = C_i + [E | A_i] [B'_i ; F], see matmul.cu).
//
// Exact modular products on the tensor cores.  Every 61-bit operand x is
// written in balanced base-2^8 digits, x = sum_d x_d 2^(8d) with
// x_d in [-128, 127] (8 digits, the top one in [0, 33]), each exactly
// representable in bf16.  For two operands the digit-pair products
// L_a * R_b (tcgen05.mma kind::f16, bf16 inputs, f32 accumulation in tensor
// memory) are summed over chunks of at most 1024 of the inner dimension:
// integers of magnitude at most 1024 * 128 * 128 = 2^24, so every partial
// f32 sum is exact; the epilogue turns each into a field element and
// multiplies it by 2^(8(a+b)) mod 2^61 - 1 (a 61-bit rotation), accumulating
// mod p:
//   L * R = sum_{chunks} sum_{a,b} 2^(8(a+b)) (L_a * R_b)   (mod p).
// (The int8 form kind::i8 is not available on sm_103a.)
//
// One CTA computes a 128 x 128 output tile of one job (or its share of the
// tile's digit-pair chains) with three roles: warp 0 loads digit-plane
// tiles with TMA, warp 1 issues the MMAs (and owns the tensor memory), warps
// 2..9 drain the accumulators.  The chains run in pairs (a, b), (a, b+1):
// both read the same left tile, so a stage holds the left tile's box and
// both right tiles' boxes side by side -- three boxes loaded per two chains'
// MMAs where separate chains load four, a quarter fewer L2 -> shared-memory
// bytes -- and the two right boxes form one 256-row operand: one M = 128,
// N = 256 MMA per 16 of the inner dimension writes both chains'
// accumulators.  A 4-stage ring of 48 KB (64 of the inner dimension per
// stage, 4 MMAs per wait) keeps three stages of loads in flight.  Two pairs
// of accumulators (all 512 tensor-memory columns) let the drain of one pair
// overlap the MMAs of the next.  Whole 2048^3 product: 12.1 ms with single
// chains, 10.65 ms with pairs as two N = 128 MMAs in a 2-stage ring of
// 96 KB, 9.5 ms here.
// Every wait is bounded: on timeout the CTA raises an error flag, stops
// issuing work, waits for what it already issued and frees its tensor
// memory.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include <cuda_bf16.h>

#include "common.cuh"

namespace spdz {

constexpr int TC_DIGITS = 8;
constexpr int TC_DIGIT_BITS = 8;
constexpr int TC_KCHUNK = 1024;       // inner length of one exact digit-pair sum
constexpr int TC_TILE = 128;          // output tile edge (M = N = 128)
constexpr int TC_KB = 64;             // K elements per TMA box (128 bytes of bf16, the swizzle span)
constexpr int TC_KSTAGE = 64;         // K elements per stage: TC_NH boxes of each tile
constexpr int TC_STAGES = 4;
constexpr int TC_NH = TC_KSTAGE / TC_KB;                      // 64-element halves of a stage
constexpr int TC_BOX_BYTES = TC_TILE * TC_KB * 2;            // one 128 x 64 bf16 box
// A stage: the left digit a's boxes (halves 0 .. TC_NH-1), then per half the
// right digits b and b+1 side by side, one 256-row operand of one MMA
constexpr int TC_STAGE_BYTES = 3 * TC_NH * TC_BOX_BYTES;
constexpr int TC_THREADS = 320;       // 10 warps
constexpr uint32_t TC_TMEM_COLS = 512;   // two chain pairs in flight, two 128-column accumulators each
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;   // bound of one pipeline wait

// ----------------------------------------------------------- digit planes
// x in [0, p) -> 8 balanced digits (low first): d = x mod 256 taken in
// [-128, 127], then x = (x - d) / 256; the top digit is in [0, 33].
__device__ __forceinline__ void balanced_digits(uint64_t x, float (&d)[TC_DIGITS]) {
    int64_t t = (int64_t)x;
#pragma unroll
    for (int j = 0; j < TC_DIGITS - 1; ++j) {
        int v = (int)(t & 255);
        if (v >= 128) v -= 256;
        d[j] = (float)v;
        t = (t - v) >> 8;
    }
    d[TC_DIGITS - 1] = (float)t;
}

// Row-major rows x cols matrix -> planes [TC_DIGITS][rows][colsp] (bf16),
// columns cols .. colsp-1 zero (colsp: cols rounded up to a multiple of 8 for
// 16-byte TMA strides).  A block takes chunks of 2048 columns of one row (one
// index division per chunk), a thread eight consecutive columns: eight loads
// in flight and one 16-byte store of eight digits per plane.
constexpr int64_t TC_DCHUNK = 2048;
// The matrices of one conversion launch (all of one shape): sources, and
// the planes each one's digits go to.
constexpr int TC_MAX_JOBS = 2 * SPDZ_MAX_PARTIES + 1;
struct DigitJobs {
    const uint64_t *x[TC_MAX_JOBS];
    int64_t ld;
    __nv_bfloat16 *planes[TC_MAX_JOBS];
    int n;
};

__global__ void k_digits_rowmajor(DigitJobs jb, int64_t rows, int64_t cols, int64_t colsp) {
    const int64_t total = rows * colsp;
    const int64_t nch = (colsp + TC_DCHUNK - 1) / TC_DCHUNK, per = rows * nch;
    for (int64_t c = blockIdx.x; c < per * jb.n; c += gridDim.x) {
        const int64_t q = c / per, cr = c - q * per;
        const int64_t r = cr / nch, k0 = (cr - r * nch) * TC_DCHUNK, k1 = min(colsp, k0 + TC_DCHUNK);
        const uint64_t *xr = jb.x[q] + r * jb.ld;
        __nv_bfloat16 *planes = jb.planes[q];
        for (int64_t c0 = k0 + 8 * (int64_t)threadIdx.x; c0 < k1; c0 += 8 * (int64_t)blockDim.x) {
            uint64_t v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = c0 + u < cols ? xr[c0 + u] : 0;
            float d[8][TC_DIGITS];
#pragma unroll
            for (int u = 0; u < 8; ++u) balanced_digits(v[u], d[u]);   // 0 gives all-zero digits
#pragma unroll
            for (int j = 0; j < TC_DIGITS; ++j) {
                uint4 w;
                __nv_bfloat162 h;
                h = __floats2bfloat162_rn(d[0][j], d[1][j]); w.x = *reinterpret_cast<const uint32_t *>(&h);
                h = __floats2bfloat162_rn(d[2][j], d[3][j]); w.y = *reinterpret_cast<const uint32_t *>(&h);
                h = __floats2bfloat162_rn(d[4][j], d[5][j]); w.z = *reinterpret_cast<const uint32_t *>(&h);
                h = __floats2bfloat162_rn(d[6][j], d[7][j]); w.w = *reinterpret_cast<const uint32_t *>(&h);
                *reinterpret_cast<uint4 *>(planes + j * total + r * colsp + c0) = w;
            }
        }
    }
}

// Row-major rows x cols matrix -> transposed planes [TC_DIGITS][cols][rowsp]
// (bf16), columns rows .. rowsp-1 of each output row zero (rowsp: a multiple
// of 8), through 64 x 32 shared-memory tiles: a thread writes two
// consecutive output columns (4-byte stores, 128 bytes per warp and plane).
__global__ void k_digits_transposed(DigitJobs jb, int64_t rows, int64_t cols, int64_t rowsp) {
    __shared__ uint64_t tile[64][33];
    const uint64_t *x = jb.x[blockIdx.z];
    __nv_bfloat16 *planes = jb.planes[blockIdx.z];
    const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 32;
    for (int i = threadIdx.y; i < 64; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? x[r * jb.ld + c] : 0;
    }
    __syncthreads();
    const int64_t total = cols * rowsp;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + 2 * threadIdx.x;   // output row c, columns r and r + 1
        if (c < cols && r < rowsp) {
            float d0[TC_DIGITS], d1[TC_DIGITS];
            balanced_digits(tile[2 * threadIdx.x][i], d0);       // rows past the matrix read 0: all-zero digits
            balanced_digits(tile[2 * threadIdx.x + 1][i], d1);
#pragma unroll
            for (int j = 0; j < TC_DIGITS; ++j)
                *reinterpret_cast<__nv_bfloat162 *>(planes + j * total + c * rowsp + r) = __floats2bfloat162_rn(d0[j], d1[j]);
        }
    }
}

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ unsigned long long tc_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(a), "r"(parity) : "memory");
    return done != 0;
}
// Bounded wait for the phase with the given parity to complete: false when
// the CTA has aborted, or (raising the abort flag) after TC_WAIT_NS.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    const uint32_t a = smem_u32(bar);
    const unsigned long long t0 = tc_now();
    for (uint32_t it = 0;; ++it) {
        if (mbar_test(a, parity)) return true;
        if ((it & 255) == 255) {
            if (*abort_flag) return false;
            if (tc_now() - t0 > TC_WAIT_NS) {
                *abort_flag = 1;
                return false;
            }
        }
    }
}
// Same bound, ignoring the abort flag (draining issued work before exit).
__device__ __forceinline__ bool mbar_drain(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    const unsigned long long t0 = tc_now();
    while (!mbar_test(a, parity))
        if (tc_now() - t0 > TC_WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(const void *p) {
    const uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;                 // start address
    d |= (uint64_t)(16 >> 4) << 16;               // leading-dimension byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;             // stride-dimension byte offset
    d |= 1ull << 46;                              // descriptor version
    d |= 2ull << 61;                              // 128-byte swizzle
    return d;
}

// bf16 x bf16 -> f32, A and B K-major, M = 128, N = 256: the two right
// digits b and b+1 of a chain pair as one 256-row operand, their
// accumulators side by side in tensor memory (256 columns).
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((2 * TC_TILE) >> 3) << 17) |
                              ((uint32_t)(TC_TILE >> 4) << 24);
static_assert(2 * TC_TILE <= 256, "N of one MMA is at most 256");

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                 "l"(a), "l"(b), "r"(TC_IDESC), "r"(accumulate)
                 : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                 "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// x * 2^e mod 2^61 - 1 for x < 2^61 - 1: rotate the 61-bit word left by e.
__device__ __forceinline__ uint64_t rot61(uint64_t x, int e) {
    return e == 0 ? x : (((x << e) | (x >> (61 - e))) & F61::P);
}

struct TcJob {
    const uint64_t *add;   // m x n, leading dimension ldo (may be null)
    uint64_t *out;
    int64_t ldo;
    int64_t m, n, k;       // k: inner length of each of the two segments
    int *err;              // set to 1 when a wait timed out
    uint64_t *part;        // nsplit > 1: [nsplit][m][n] partial sums, combined by k_tc_combine
    int nsplit;            // CTAs per output tile (blockIdx.z: which share of the digit-pair chains)
};

// maps: left segment 0, left segment 1, right segment 0, right segment 1
// (3-D: x = inner index, y = row of the K-major tile, z = digit).
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_gemm(const __grid_constant__ CUtensorMap L0,
                                                           const __grid_constant__ CUtensorMap L1,
                                                           const __grid_constant__ CUtensorMap R0,
                                                           const __grid_constant__ CUtensorMap R1, TcJob job) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full_bar[TC_STAGES], empty_bar[TC_STAGES], acc_full[2], acc_empty[2], done_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_flag;
    __shared__ int issued_g, consumed_g;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.y * TC_TILE, col0 = (int64_t)blockIdx.x * TC_TILE;
    // chain pairs: (segment, inner chunk of TC_KCHUNK, digit a, digits
    // 2 bp and 2 bp + 1), bp fastest; this CTA's share [c0, c1) of the
    // tile's pairs
    constexpr int BPAIRS = TC_DIGITS / 2;
    const int nchunks = (int)((job.k + TC_KCHUNK - 1) / TC_KCHUNK);
    const int per_chunk = TC_DIGITS * BPAIRS;
    const int npairs = 2 * nchunks * per_chunk;
    auto chain_kblocks = [&](int kc) {
        const int64_t len = min((int64_t)TC_KCHUNK, job.k - (int64_t)kc * TC_KCHUNK);
        return (int)((len + TC_KSTAGE - 1) / TC_KSTAGE);
    };
    const int c0 = (int)((int64_t)npairs * blockIdx.z / job.nsplit), c1 = (int)((int64_t)npairs * (blockIdx.z + 1) / job.nsplit);
    const int chains = c1 - c0;   // chain pairs of this CTA

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 8);        // one arrival per epilogue warp
        }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        issued_g = consumed_g = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_sh;

    if (warp == 0) {
        // ---------------------------------------------------------- TMA
        if (lane == 0) {
            int g = 0;
            for (int ci = 0; ci < chains && !abort_flag; ++ci) {
                const int c = c0 + ci;
                const int seg = c / (nchunks * per_chunk), kc = (c / per_chunk) % nchunks;
                const int a = (c / BPAIRS) % TC_DIGITS, b = 2 * (c % BPAIRS);
                const CUtensorMap *Lm = seg == 0 ? &L0 : &L1, *Rm = seg == 0 ? &R0 : &R1;
                const int kblocks = chain_kblocks(kc), kbase = kc * TC_KCHUNK;
                for (int kb = 0; kb < kblocks; ++kb, ++g) {
                    const int s = g % TC_STAGES;
                    const uint32_t ph = (uint32_t)(g / TC_STAGES) & 1u;
                    if (g >= TC_STAGES && !mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag)) break;
                    // left digit a's halves first; per half h the right
                    // digits b and b + 1 in adjacent boxes
                    unsigned char *st = smem + (size_t)s * TC_STAGE_BYTES;
                    mbar_expect_tx(&full_bar[s], TC_STAGE_BYTES);
#pragma unroll
                    for (int h = 0; h < TC_NH; ++h) {
                        const int kx = kbase + kb * TC_KSTAGE + h * TC_KB;
                        tma_load_3d(st + h * TC_BOX_BYTES, Lm, kx, (int)row0, a, &full_bar[s]);
                        tma_load_3d(st + (TC_NH + 2 * h) * TC_BOX_BYTES, Rm, kx, (int)col0, b, &full_bar[s]);
                        tma_load_3d(st + (TC_NH + 2 * h + 1) * TC_BOX_BYTES, Rm, kx, (int)col0, b + 1, &full_bar[s]);
                    }
                    issued_g = g + 1;
                }
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA
        if (lane == 0) {
            int g = 0;
            for (int ci = 0; ci < chains && !abort_flag; ++ci) {
                const int ab = ci & 1;
                const uint32_t acc_ph = (uint32_t)(ci >> 1) & 1u;
                if (ci >= 2 && !mbar_wait(&acc_empty[ab], acc_ph ^ 1u, &abort_flag)) break;
                tc_fence_after();
                // accumulators of digits b and b + 1: columns [256 ab, +128) and [256 ab + 128, +128),
                // written by one N = 256 MMA at d0
                const uint32_t d0 = tmem_base + (uint32_t)(ab * 2 * TC_TILE);
                const int kblocks = chain_kblocks(((c0 + ci) / per_chunk) % nchunks);
                bool ok = true;
                for (int kb = 0; kb < kblocks; ++kb, ++g) {
                    const int s = g % TC_STAGES;
                    const uint32_t ph = (uint32_t)(g / TC_STAGES) & 1u;
                    if (!mbar_wait(&full_bar[s], ph, &abort_flag)) { ok = false; break; }
                    consumed_g = g + 1;
                    tc_fence_after();
                    const unsigned char *st = smem + (size_t)s * TC_STAGE_BYTES;
#pragma unroll
                    for (int k16 = 0; k16 < TC_KSTAGE / 16; ++k16) {
                        const int h = k16 / (TC_KB / 16), kk = k16 % (TC_KB / 16);
                        const uint64_t da = smem_desc(st + h * TC_BOX_BYTES),
                                       db = smem_desc(st + (TC_NH + 2 * h) * TC_BOX_BYTES);
                        const uint32_t acc = (kb | k16) != 0;
                        // one MMA for both chains: rows 0-127 of the right
                        // operand are digit b (into d0), 128-255 digit b+1 (d1)
                        mma_bf16(d0, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), acc);
                    }
                    mma_commit(&empty_bar[s]);     // frees the stage once these MMAs have read it
                }
                if (!ok) break;
                mma_commit(&acc_full[ab]);         // the accumulator is complete
            }
            // every MMA issued above has completed once this commit arrives
            mma_commit(&done_bar);
            if (!mbar_drain(&done_bar, 0)) abort_flag = 1;
        }
    } else {
        // ----------------------------------------------------- epilogue
        const int ew = warp - 2;                    // 0..7
        const int quad = warp & 3;                  // TMEM lanes 32*quad .. +31 (rows)
        const int half = ew >> 2;                   // columns 64*half .. +63
        const int64_t row = row0 + quad * 32 + lane;
        // Each accumulator entry v is an integer with |v| <= 2^24: it is
        // taken as v + 2^24 >= 0 and the offsets, sum_c 2^24 2^(e_c) mod p,
        // come off once at the end.  Sums are kept below 2^61 + 2 by one
        // fold per addition (2^61 == 1) and reduced at the end.
        uint64_t sum[64], off = 0;
#pragma unroll
        for (int j = 0; j < 64; ++j) sum[j] = 0;
        for (int ci = 0; ci < chains; ++ci) {
            const int c = c0 + ci;
            const int ab = ci & 1;
            const uint32_t acc_ph = (uint32_t)(ci >> 1) & 1u;
            if (!mbar_wait(&acc_full[ab], acc_ph, &abort_flag)) break;
            tc_fence_after();
            const int a = (c / BPAIRS) % TC_DIGITS, b0 = 2 * (c % BPAIRS);
#pragma unroll 1
            for (int sub = 0; sub < 2; ++sub) {
                const int e = (TC_DIGIT_BITS * (a + b0 + sub)) % 61;
                off = F61::add(off, rot61(1ull << 24, e));
                const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) +
                                       (uint32_t)((2 * ab + sub) * TC_TILE + half * 64);
                // for e <= 36, u * 2^e <= 2^61 needs no wrap: a plain shift
                auto drain = [&](auto nowrap) {
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        uint32_t r[32];
                        tmem_ld32(taddr + (uint32_t)(q * 32), r);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int32_t v = __float2int_rn(__uint_as_float(r[j]));    // exact, |v| <= 2^24
                            const uint64_t u = (uint64_t)(uint32_t)(v + (1 << 24));       // [0, 2^25]
                            const uint64_t t = sum[q * 32 + j] + (decltype(nowrap)::value ? u << e : rot61(u, e));
                            sum[q * 32 + j] = (t & F61::P) + (t >> 61);                   // < 2^61 + 2
                        }
                    }
                };
                if (e <= 36) drain(std::true_type{});
                else drain(std::false_type{});
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[ab]);
        }
#pragma unroll
        for (int j = 0; j < 64; ++j) {
            uint64_t v = sum[j];
            v = v >= F61::P ? v - F61::P : v;                 // canonical (v <= p + 1 before)
            sum[j] = F61::sub(v, off);
        }
        if (!abort_flag && row < job.m) {
            if (job.nsplit == 1) {
#pragma unroll
                for (int j = 0; j < 64; ++j) {
                    const int64_t col = col0 + half * 64 + j;
                    if (col < job.n) {
                        uint64_t v = sum[j];
                        if (job.add) v = F61::add(v, job.add[row * job.ldo + col]);
                        job.out[row * job.ldo + col] = v;
                    }
                }
            } else {
                uint64_t *prow = job.part + ((int64_t)blockIdx.z * job.m + row) * job.n;
#pragma unroll
                for (int j = 0; j < 64; ++j) {
                    const int64_t col = col0 + half * 64 + j;
                    if (col < job.n) prow[col] = sum[j];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (abort_flag && threadIdx.x == 0) {
        // loads issued but never consumed must land before the CTA exits
        for (int g = consumed_g; g < issued_g; ++g) mbar_drain(&full_bar[g % TC_STAGES], (uint32_t)(g / TC_STAGES) & 1u);
        atomicExch(job.err, 1);
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TC_TMEM_COLS) : "memory");
    }
}

// out = add + sum of the nsplit partial tiles, mod p (elementwise).  A block
// walks whole rows (no index division); the partials are read once.
__global__ void k_tc_combine(const uint64_t *part, int nsplit, int64_t m, int64_t n, const uint64_t *add, uint64_t *out,
                             int64_t ldo) {
    const int64_t total = m * n;
    for (int64_t r = blockIdx.x; r < m; r += gridDim.x) {
        const unsigned long long *pr = reinterpret_cast<const unsigned long long *>(part) + r * n;
#pragma unroll 4
        for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
            uint64_t v = add ? add[r * ldo + c] : 0;
            for (int q = 0; q < nsplit; ++q) v = F61::add(v, __ldcs(pr + q * total + c));
            out[r * ldo + c] = v;
        }
    }
}

// ------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// Tensor map over digit planes [9][rows][inner] (bf16, inner contiguous),
// boxes of 64 inner x 128 rows x 1 digit, 128-byte swizzle; reads outside
// the matrix return zero.
static bool make_map(CUtensorMap *map, const void *planes, int64_t rows, int64_t inner) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, (cuuint64_t)TC_DIGITS};
    const cuuint64_t strides[2] = {(cuuint64_t)inner * 2, (cuuint64_t)(inner * rows * 2)};
    const cuuint32_t box[3] = {TC_KB, TC_TILE, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(planes), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TcWorkspace {
    void *p = nullptr;
    size_t bytes = 0;
};

int matmul_tensor(spdz_ctx *ctx, const uint64_t *E, const uint64_t *Fm, const uint64_t *Rfold, const spdz_buf *A,
                  const spdz_buf *C, const spdz_buf *Z, int64_t m, int64_t k, int64_t n) {
    if (m <= 0 || n <= 0 || k <= 0 || k > 2048)
        return set_err(ctx, SPDZ_ERR_ARG, "matmul tensor: inner length must be 1..2048 (exact f32 sums)");
    const int NPn = ctx->n;
    const int64_t kp = (k + 7) / 8 * 8;    // padded inner length: 16-byte TMA strides
    const size_t plane_l = (size_t)TC_DIGITS * m * kp * 2, plane_r = (size_t)TC_DIGITS * n * kp * 2;
    // digits of E and of every A block (left), of every folded right block and of F (right, transposed)
    // CTAs per output tile: the smallest split (at most 8) whose last wave of
    // one-CTA-per-SM launches is at least 95 % full
    const int64_t tiles = ((n + TC_TILE - 1) / TC_TILE) * ((m + TC_TILE - 1) / TC_TILE);
    int nsplit = 1;
    {
        double best = 0.0;
        for (int ns = 1; ns <= 8; ++ns) {
            const int64_t ctas = tiles * ns, waves = (ctas + ctx->sm_count - 1) / ctx->sm_count;
            const double fill = (double)ctas / (double)(waves * ctx->sm_count);
            if (fill > best + 1e-9) { best = fill; nsplit = ns; }
            if (fill >= 0.95) break;
        }
    }
    const size_t part_bytes = nsplit > 1 ? (size_t)nsplit * m * n * sizeof(uint64_t) : 0;
    const size_t need = plane_l * (1 + 2 * NPn) + plane_r * (1 + 2 * NPn) + part_bytes + 512;
    static std::mutex mu;
    static TcWorkspace ws;   // shared by contexts of this process, grown on demand
    std::lock_guard<std::mutex> g(mu);
    if (need > ws.bytes) {
        cudaStreamSynchronize(ctx->stream);
        if (ws.p) cudaFree(ws.p);
        ws.p = nullptr;
        ws.bytes = 0;
        if (cudaMalloc(&ws.p, need) != cudaSuccess) return set_err(ctx, SPDZ_ERR_OOM, "matmul tensor: workspace");
        ws.bytes = need;
    }
    unsigned char *base = (unsigned char *)ws.p;
    int *err = (int *)base;
    __nv_bfloat16 *dE = (__nv_bfloat16 *)(base + 256);
    __nv_bfloat16 *dA = (__nv_bfloat16 *)((unsigned char *)dE + plane_l);
    __nv_bfloat16 *dF = (__nv_bfloat16 *)((unsigned char *)dA + plane_l * 2 * NPn);
    __nv_bfloat16 *dR = (__nv_bfloat16 *)((unsigned char *)dF + plane_r);
    uint64_t *dP = (uint64_t *)((((uintptr_t)((unsigned char *)dR + plane_r * 2 * NPn)) + 255) & ~(uintptr_t)255);
    cudaMemsetAsync(err, 0, sizeof(int), ctx->stream);
    const int gb = 4 * ctx->sm_count;
    // every left matrix (E, then A_i values and MACs) in one launch, every
    // right matrix (F, then the folded B_i) in another
    DigitJobs jl{}, jr{};
    jl.n = jr.n = 1 + 2 * NPn;
    jl.ld = k;
    jr.ld = n;
    jl.x[0] = E;
    jl.planes[0] = dE;
    jr.x[0] = Fm;
    jr.planes[0] = dF;
    for (int w = 0; w < 2; ++w)
        for (int i = 0; i < NPn; ++i) {
            jl.x[1 + w * NPn + i] = (const uint64_t *)(w == 0 ? A->val : A->mac) + (int64_t)i * A->stride;
            jl.planes[1 + w * NPn + i] = (__nv_bfloat16 *)((unsigned char *)dA + plane_l * (w * NPn + i));
        }
    for (int j = 0; j < 2 * NPn; ++j) {
        jr.x[1 + j] = Rfold + (int64_t)j * k * n;
        jr.planes[1 + j] = (__nv_bfloat16 *)((unsigned char *)dR + plane_r * j);
    }
    const int gd = (int)std::min<int64_t>(jl.n * m * ((kp + TC_DCHUNK - 1) / TC_DCHUNK), 8 * (int64_t)ctx->sm_count);
    k_digits_rowmajor<<<gd, 256, 0, ctx->stream>>>(jl, m, k, kp);
    // the transposed kernel covers output columns 0 .. kp-1 (padding included)
    dim3 tg((unsigned)((n + 31) / 32), (unsigned)((kp + 63) / 64), (unsigned)jr.n), tb(32, 8);
    k_digits_transposed<<<tg, tb, 0, ctx->stream>>>(jr, k, n, kp);
    if (int rc = check_launch(ctx, "matmul tensor digits")) return rc;
    const size_t smem = (size_t)TC_STAGES * TC_STAGE_BYTES + 1024;
    cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    CUtensorMap mE, mF;
    if (!make_map(&mE, dE, m, kp) || !make_map(&mF, dF, n, kp))
        return set_err(ctx, SPDZ_ERR_CUDA, "matmul tensor: tensor map encoding failed");
    dim3 grid((unsigned)((n + TC_TILE - 1) / TC_TILE), (unsigned)((m + TC_TILE - 1) / TC_TILE), (unsigned)nsplit);
    for (int w = 0; w < 2; ++w)
        for (int i = 0; i < NPn; ++i) {
            const int j = w * NPn + i;
            CUtensorMap mA, mR;
            if (!make_map(&mA, (unsigned char *)dA + plane_l * j, m, kp) || !make_map(&mR, (unsigned char *)dR + plane_r * j, n, kp))
                return set_err(ctx, SPDZ_ERR_CUDA, "matmul tensor: tensor map encoding failed");
            TcJob job;
            job.add = (const uint64_t *)(w == 0 ? C->val : C->mac) + (int64_t)i * C->stride;
            job.out = (uint64_t *)(w == 0 ? Z->val : Z->mac) + (int64_t)i * Z->stride;
            job.ldo = n;
            job.m = m;
            job.n = n;
            job.k = kp;
            job.err = err;
            job.part = dP;
            job.nsplit = nsplit;
            // left [E | A_j], right [Rfold_j ; F] (transposed: rows are output columns)
            k_tc_gemm<<<grid, TC_THREADS, smem, ctx->stream>>>(mE, mA, mR, mF, job);
            if (int rc = check_launch(ctx, "matmul tensor gemm")) return rc;
            if (nsplit > 1) {
                k_tc_combine<<<gb, 256, 0, ctx->stream>>>(dP, nsplit, m, n, job.add, job.out, job.ldo);
                if (int rc = check_launch(ctx, "matmul tensor combine")) return rc;
            }
        }
    int herr = 0;
    cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (int rc = check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "matmul tensor")) return rc;
    if (herr) return set_err(ctx, SPDZ_ERR_TIMEOUT, "matmul tensor: a pipeline wait timed out");
    return SPDZ_OK;
}

}  // namespace spdz
