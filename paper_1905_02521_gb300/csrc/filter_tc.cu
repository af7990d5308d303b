// filter_tc.cu -- the coloured-noise filter (Eqs. 6-7) as a blocked Toeplitz
// GEMM on the sm_103a tensor cores (tcgen05, BF16 operands, FP32 accumulation
// in tensor memory).
//
// For one 256-step block b and one system, eta[j][d] = sum_tau X[d][tau] T[tau][j]:
//   X[d][tau] = xi(256 b - K_e + tau, d)   (white noise, the ring of BF16 blocks)
//   T[tau][j] = h_|j - tau + K_e|          (Toeplitz band of the taps; 0 outside |k| <= K)
// with K_e = 256 K_b the padded half length, tau < 256 (2 K_b + 1).  M = 128 dofs
// per CTA, N = 256 steps, K = 256 (2 K_b + 1) streamed in 64-wide chunks.
//
// Roles in one CTA of 128 threads: thread 0 issues the TMA loads (A tile
// 128x64 and B tile 256x64, 128-byte swizzle), thread 32 issues tcgen05.mma
// (M128 N256 K16) and commits each stage back to its producer barrier; all four
// warps then read the 128x256 FP32 accumulator from tensor memory and store
// eta[j][dof] coalesced.  Every mbarrier wait is bounded by a clock budget;
// on timeout the CTA raises an error bit, drains, frees its tensor memory and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "qtb_dev.cuh"
#include "qtb_kernels.cuh"

namespace qtb {

namespace tc {

constexpr int BM = 128, BN = 256, BK = 64;          // tile, K chunk (BF16: 64 x 2 B = 128 B rows)
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;                 // 16 KB
constexpr int B_BYTES = BN * BK * 2;                 // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /* align */ + 256 /* barriers */;
constexpr long long WAIT_BUDGET = 4000000000LL;      // clock cycles (~2 s) per wait

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: returns false after the clock budget is spent
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > WAIT_BUDGET) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *map, unsigned bar, int c0, int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(dst), "l"((unsigned long long)map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((addr & 0x3FFFF) >> 4);            // start address
    d |= (unsigned long long)1 << 16;                            // leading byte offset (unused for SW128 K-major)
    d |= (unsigned long long)(1024 >> 4) << 32;                  // stride byte offset
    d |= (unsigned long long)1 << 46;                            // descriptor version (sm_100 family)
    d |= (unsigned long long)2 << 61;                            // SWIZZLE_128B
    return d;
}

// instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major, M = 128, N = 256
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N)
{
    return (1u << 4)                  // D format F32
           | (1u << 7)                // A format BF16
           | (1u << 10)               // B format BF16
           | ((unsigned)(N >> 3) << 17)
           | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, unsigned long long adesc, unsigned long long bdesc,
                                         unsigned idesc, unsigned accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32])
{
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

}  // namespace tc

// grid = number of 128-dof tiles; block = 128 threads
__global__ void __launch_bounds__(128, 1)
k_filter_tc(Dev d, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            const int2 *__restrict__ tiles /* (system, first dof within system) */)
{
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned stage buffers (required by the 128-byte swizzle)
    const unsigned base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (base - smem_u32(smem_raw));
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(gbase + STAGES * STAGE_BYTES);
    // bars[0..S): full, bars[S..2S): empty, bars[2S]: done; then tmem address and abort flag
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(bars + 2 * STAGES + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int2 tile = tiles[blockIdx.x];
    const DSys S = d.sys[tile.x];
    const int nchunks = d.nslots * (kBlockSteps / BK);
    const long long blk = d.clock[0];
    const unsigned full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done = smem_u32(bars + 2 * STAGES);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {  // allocate 256 TMEM columns (128 lanes x 256 x 32-bit accumulator)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;

    if (threadIdx.x == 0) {
        // ---------------- TMA producer
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % STAGES;
            if (c >= STAGES && !mbar_wait(empty0 + 8 * s, ((c / STAGES) - 1) & 1)) {
                *abort_flag = 1;
                break;
            }
            if (*abort_flag) break;
            const unsigned sa = base + s * STAGE_BYTES, sb = sa + A_BYTES;
            mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
            // ring block of this chunk: b - K_b + c/4, slot = that block mod nslots
            const long long rb = blk - d.Kb + c / (kBlockSteps / BK);
            const int slot = (int)(rb - floor_div(rb, d.nslots) * d.nslots);
            tma_load_3d(sa, &tmA, full0 + 8 * s, (c % (kBlockSteps / BK)) * BK, S.dof0 + tile.y, slot);
            tma_load_3d(sb, &tmB, full0 + 8 * s, c * BK, 0, tile.x);
        }
    } else if (threadIdx.x == 32) {
        // ---------------- MMA issuer
        const unsigned idesc = idesc_bf16(BM, BN);
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % STAGES;
            if (!mbar_wait(full0 + 8 * s, (c / STAGES) & 1)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const unsigned sa = base + s * STAGE_BYTES, sb = sa + A_BYTES;
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)  // K = 16 per instruction, 32 bytes along the swizzled row
                mma_bf16(tmem, smem_desc(sa + 32 * k), smem_desc(sb + 32 * k), idesc, (c > 0 || k > 0) ? 1u : 0u);
            mma_commit(empty0 + 8 * s);  // stage s may be refilled once these MMAs have read it
        }
        mma_commit(done);  // accumulator complete (tracks every MMA issued above)
    }
    __syncwarp();
    // ---------------- epilogue: TMEM -> registers -> eta[j][dof]
    const bool ok_t = mbar_wait(done, 0);
    __syncwarp();
    tc_fence_after();
    const bool ok = __all_sync(0xffffffffu, ok_t && !*abort_flag);
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(d.err, (unsigned)ERR_TIMEOUT_TC);
    } else {
        float *eta = reinterpret_cast<float *>(d.eta);
        const int row = warp * 32 + lane;  // dof within the tile (TMEM lane)
        const int dofl = tile.y + row;
        const bool valid = dofl < 3 * S.N * S.P;
        const size_t col0 = (size_t)S.dof0 + dofl;
#pragma unroll 1
        for (int j0 = 0; j0 < BN; j0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)j0, v);
#pragma unroll
            for (int k = 0; k < 32; ++k) eta[(size_t)(j0 + k) * d.Dtot + col0] = valid ? v[k] : 0.0f;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

// Toeplitz band of each system's taps in BF16: Bt[s][j][tau] = h_|j - tau + K_e| (0 if > K_s).
// grid = (Ktot / 256, 256 rows j, nsys), block 256
__global__ void k_build_toeplitz(Dev d, __nv_bfloat16 *Bt, int Ktot, int Ke)
{
    const DSys S = d.sys[blockIdx.z];
    const int j = blockIdx.y;
    const int tau = blockIdx.x * blockDim.x + threadIdx.x;
    if (tau >= Ktot) return;
    const int k = j - tau + Ke;
    const int ka = k < 0 ? -k : k;
    const float *h = reinterpret_cast<const float *>(d.tapsR) + S.taps0;
    const float v = (ka <= S.K) ? h[ka] : 0.0f;
    Bt[((size_t)blockIdx.z * 256 + j) * Ktot + tau] = __float2bfloat16_rn(v);
}

cudaError_t filter_tc_prepare()
{
    return cudaFuncSetAttribute(k_filter_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
}

void launch_build_toeplitz(const Dev &d, void *Bt, int Ktot, int Ke, cudaStream_t st)
{
    dim3 grid((unsigned)((Ktot + 255) / 256), 256u, (unsigned)d.nsys);
    k_build_toeplitz<<<grid, 256, 0, st>>>(d, reinterpret_cast<__nv_bfloat16 *>(Bt), Ktot, Ke);
}

void launch_filter_tc(const Dev &d, const void *tmapA, const void *tmapB, int n_mtiles, const int *mtile_sys,
                      cudaStream_t st)
{
    const CUtensorMap *A = reinterpret_cast<const CUtensorMap *>(tmapA);
    const CUtensorMap *B = reinterpret_cast<const CUtensorMap *>(tmapB);
    k_filter_tc<<<n_mtiles, 128, tc::SMEM_BYTES, st>>>(d, *A, *B, reinterpret_cast<const int2 *>(mtile_sys));
}

}  // namespace qtb
