// tcgen05 engine of the surrogate's 32 -> 32 convolutions (sm_103a).
//
// Both kernels compute the periodic 3x3x3 convolution as an implicit GEMM on
// the 5th-generation tensor cores: D[128 voxels x N] (FP32, in tensor memory)
// += A[128 x 16] (BF16 activations, shared memory) x B[16 x N] (BF16 weights,
// shared memory), over the taps and 2 K-steps of 16 input channels. The
// weights use the no-swizzle K-major core-matrix layout (a core matrix is
// 8 rows x 16 bytes stored as 128 contiguous bytes; the descriptor gives the
// distance of core matrices adjacent along K (leading byte offset, 128 B) and
// along N (stride byte offset, 512 B)).
//
// conv_ring_kernel (Z a multiple of 128): a persistent, warp-specialised
// pipeline. A work unit is a run of output rows (b, x, y = ys .. ye-1,
// z0 .. z0+127); the 128 voxels of a row are the MMA's M. The kernel walks the
// INPUT rows y' = ys-1 .. ye: a ring slot holds input row (b, x-1 .. x+1, y')
// as [dx][z][32 ci] with 64-byte z rows in the 64-byte swizzle layout, exactly
// as TMA writes it (row 16 + i holds z0 + i, rows 0..15 and 144..159 the
// periodic halo), so the operand of tap dz starts dz rows later and its second
// K-step 32 bytes on. One input row feeds output rows y'+1, y', y'-1 (dy = -1,
// 0, +1): the weights of the three dy are stacked along N = 96, so each input
// row costs 18 MMAs (3 dx x 3 dz x 2 K-steps) into three consecutive
// accumulator blocks of a 16-block ring (32 columns per output row, descending
// with the row so that the three blocks are adjacent; where they wrap past
// column 511 each MMA splits into N = 64 + 32). Blocks start at zero and only
// accumulate; an output row is complete after its third input row.
//   warp 0      producer: per slot 9 TMA loads (per dx the 128 rows z0 ..
//               and two 16-row halo boxes at (z0-16) mod Z, (z0+128) mod Z);
//               a full mbarrier per slot; a slot is refilled once the
//               commit of the row it held (below) has fired
//   warp 1      MMA issuer: the warp walks the schedule converged; lane 0 waits,
//               issues (predicated, not branched) and commits once per input
//               row, on the block of the output row that row completes (which
//               also frees the row's slot)
//   warps 2..9  epilogue: each warp reads 16 columns of its 32 lanes of a
//               completed block (tcgen05.ld), zeroes them (tcgen05.st), frees
//               the block, applies bias and the fused epilogue and stores BF16
//               channels-last; the two partial rows at each end of a unit are
//               dropped
// conv_tc_kernel (Z a multiple of 64): an unpipelined variant per tile of
// 2 rows x 64 z with three dz-shifted no-swizzle halo copies, N = 32.
//
// Every mbarrier wait is bounded (about 1 s); a wait that runs out sets the
// device flag g_tc_timeout, makes the other roles stop, waits (bounded) for
// its own copies and MMAs in flight, frees the tensor memory and returns. The
// host reads the flag with tc_take_timeout.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/evx_nn.h"
#include "evx_nn_common.cuh"

namespace evxnn {

__device__ int g_tc_timeout;

// ------------------------------------------------------------- primitives
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version (sm_100 family); no swizzle, base offset 0
    return d;
}

// K-major operand in the 64-byte swizzle layout (rows of 64 bytes, 16-byte
// chunks permuted by address bits 7..8 within 512-byte atoms): rows 64 bytes
// apart, 8-row groups 512 bytes apart. The permutation follows the absolute
// shared-memory address (as TMA applies it), so a start moved by whole rows
// or by 32 bytes addresses the same stored layout.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) { return sdesc(saddr, 16, 512) | (4ull << 61); }

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, N, M
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// the same MMA executed by the whole (converged) warp and issued by lane 0 alone
// through an instruction predicate: no divergent branch around the issue, which
// on sm_103a took the ring's 18-MMA issue sequence from about 1,570 to 1,200 cycles
__device__ __forceinline__ void tc_mma_lane0(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc) {
    asm volatile(
        "{\n .reg .pred p, q;\n .reg .u32 l;\n mov.u32 l, %%laneid;\n setp.eq.u32 p, l, 0;\n"
        " setp.ne.b32 q, %4, 0;\n @p tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(1)
        : "memory");
}

// arrive on bar once every MMA this thread issued before has completed
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait (about 2 s) for the phase of the given parity
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (clock64() - t0 > (1LL << 32)) return false;
    }
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load4(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// bias + fused epilogue on NCH (a multiple of 8) channels c0 .. of voxel vox,
// r = FP32 accumulator bits, bias = the NCH biases (registers); BF16 stores
// of 16 bytes
template <int EPI, int NCH>
__device__ __forceinline__ void epilogue_store(const ConvArgs& a, long long vox, int c0, const uint32_t* r,
                                               const float* bias) {
    const long long o = vox * 32 + c0;
#pragma unroll
    for (int q = 0; q < NCH / 8; ++q) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[q * 8 + j]) + bias[q * 8 + j];
        uint4 outw;
        __nv_bfloat162* ow = reinterpret_cast<__nv_bfloat162*>(&outw);
        if (EPI == EVX_NN_EPI_GELU) {
            uint4 pw;
            __nv_bfloat162* pp = reinterpret_cast<__nv_bfloat162*>(&pw);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                pp[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                ow[j] = __floats2bfloat162_rn(gelu(v[2 * j]), gelu(v[2 * j + 1]));
            }
            if (a.pre) *reinterpret_cast<uint4*>(a.pre + o + q * 8) = pw;  // NULL: inference, not kept
        } else if (EPI == EVX_NN_EPI_GELU_BWD) {
            const uint4 pw = *reinterpret_cast<const uint4*>(a.pre + o + q * 8);
            const __nv_bfloat162* pp = reinterpret_cast<const __nv_bfloat162*>(&pw);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 pf = __bfloat1622float2(pp[j]);
                ow[j] = __floats2bfloat162_rn(v[2 * j] * gelu_grad(pf.x), v[2 * j + 1] * gelu_grad(pf.y));
            }
        } else if (EPI == EVX_NN_EPI_RESID) {
            const uint4 rw = *reinterpret_cast<const uint4*>(a.res + o + q * 8);
            const __nv_bfloat162* rp = reinterpret_cast<const __nv_bfloat162*>(&rw);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 rf = __bfloat1622float2(rp[j]);
                ow[j] = __floats2bfloat162_rn(v[2 * j] + rf.x, v[2 * j + 1] + rf.y);
            }
        } else if (EPI == EVX_NN_EPI_RESID32) {  // FP32 stream in a.pre, updated in place
            float4* sp = reinterpret_cast<float4*>(reinterpret_cast<float*>(a.pre) + o + q * 8);
            float4 s0 = sp[0], s1 = sp[1];
            s0.x += v[0], s0.y += v[1], s0.z += v[2], s0.w += v[3];
            s1.x += v[4], s1.y += v[5], s1.z += v[6], s1.w += v[7];
            sp[0] = s0;
            sp[1] = s1;
            ow[0] = __floats2bfloat162_rn(s0.x, s0.y);
            ow[1] = __floats2bfloat162_rn(s0.z, s0.w);
            ow[2] = __floats2bfloat162_rn(s1.x, s1.y);
            ow[3] = __floats2bfloat162_rn(s1.z, s1.w);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) ow[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        }
        *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.out) + o + q * 8) = outw;
    }
}

// EVX_NN_EPI_RESID32 for one epilogue warp: 32 voxels vox0 .. vox0 + 31 (lane = voxel
// of acc) x 16 channels c0 ... The sums are staged in shared memory ([voxel][16],
// 16-byte chunk c of row v at chunk c ^ ((v >> 1) & 3): conflict-free both ways) and
// the stream is read and written with lane l on voxel l / 4 + 8 i, channels
// c0 + 4 (l % 4) ..: every instruction covers 8 whole 64-byte row pieces instead of
// one 16-byte piece of 32 rows.
__device__ __forceinline__ void resid32_staged(const ConvArgs& a, long long vox0, int c0, const uint32_t* acc,
                                               const float* bias, float* stg, int lane) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4*>(stg + lane * 16 + 4 * (q ^ ((lane >> 1) & 3))) =
            make_float4(__uint_as_float(acc[4 * q]) + bias[4 * q], __uint_as_float(acc[4 * q + 1]) + bias[4 * q + 1],
                        __uint_as_float(acc[4 * q + 2]) + bias[4 * q + 2],
                        __uint_as_float(acc[4 * q + 3]) + bias[4 * q + 3]);
    __syncwarp();
    const int c = lane & 3;
    float4 s[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int v = (lane >> 2) + 8 * i;
        s[i] = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(a.pre) + (vox0 + v) * 32 + c0 + 4 * c);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int v = (lane >> 2) + 8 * i;
        const float4 d = *reinterpret_cast<const float4*>(stg + v * 16 + 4 * (c ^ ((v >> 1) & 3)));
        s[i].x += d.x, s[i].y += d.y, s[i].z += d.z, s[i].w += d.w;
        const long long o = (vox0 + v) * 32 + c0 + 4 * c;
        *reinterpret_cast<float4*>(reinterpret_cast<float*>(a.pre) + o) = s[i];
        uint2 ob;
        __nv_bfloat162 lo = __floats2bfloat162_rn(s[i].x, s[i].y), hi = __floats2bfloat162_rn(s[i].z, s[i].w);
        ob.x = *reinterpret_cast<uint32_t*>(&lo);
        ob.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(a.out) + o) = ob;
    }
    __syncwarp();  // staging reads done before the next row overwrites it
}

// weights [t][co][ci] -> core-matrix layout [t][co/8][ci/8][8 co][8 ci]
__device__ __forceinline__ void stage_weights(unsigned char* swb, const __nv_bfloat16* w, int nthreads) {
    for (int e = threadIdx.x; e < 27 * 32 * 4; e += nthreads) {  // 16-byte pieces (t, co, ci/8)
        const int cig = e & 3, co = (e >> 2) & 31, t = e >> 7;
        const uint4 v = *reinterpret_cast<const uint4*>(w + (t * 32 + co) * 32 + cig * 8);
        *reinterpret_cast<uint4*>(swb + (((t * 4 + (co >> 3)) * 4 + cig) * 8 + (co & 7)) * 16) = v;
    }
}

// ----------------------------------------------- pipelined scatter kernel
namespace ring {
constexpr int ZT = 128;                    // voxels per output row tile (MMA M)
constexpr int RZ = 160;                    // z rows (64 bytes each) per x-row run: z0 + i at row 16 + i
constexpr int RUN = RZ * 64;               // bytes per run (a multiple of 1024)
constexpr int NS = 5;                      // ring slots (one input row each)
constexpr int SLOT = 3 * RUN;              // bytes per slot: runs for x-1, x, x+1
constexpr int WB = 9 * 12 * 4 * 128;       // staged weights: [dx][dz][n/8 (12)][ci/8][8 n][8 ci]
constexpr int NBLK = 16;                   // accumulator blocks of 32 columns (a ring over output rows)
constexpr int NEPI = 8;                    // epilogue warps
constexpr int NTH = (2 + NEPI) * 32;
constexpr int BAR = WB + NS * SLOT;        // barriers: full[NS], tfull[NBLK], tempty[NBLK]
constexpr int STG = (BAR + 8 * (NS + 2 * NBLK) + 16 + 15) & ~15;  // after the tensor-memory slot and abort flag
constexpr int STG_WARP = 32 * 16 * 4;      // per epilogue warp: [32 voxels][16 channels] FP32 staging
constexpr int SMEM = STG + NEPI * STG_WARP + 1024;  // + alignment
constexpr uint32_t SLOT_TX = SLOT;         // TMA bytes per slot
constexpr long long WAIT_BUDGET = 1LL << 31;
}  // namespace ring

struct RingArgs {
    ConvArgs a;
    int nzc;     // Z / 128
    int nseg;    // y segments per (b, x, z-chunk) column
    int nunits;  // B * X * nzc * nseg
};

// non-blocking probe of a phase (no suspend, unlike try_wait)
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait that also gives up once another role has aborted; a phase that has
// already completed is seen by the non-blocking probe first
__device__ __forceinline__ bool ring_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > ring::WAIT_BUDGET) {
            *abort_flag = 1;
            atomicExch(&g_tc_timeout, 1);
            return false;
        }
    }
}

// unit u -> column bx = b * X + x, z-chunk start z0, output rows ys .. ye-1
__device__ __forceinline__ void ring_unit(const RingArgs& r, int u, int& bx, int& z0, int& ys, int& ye) {
    const int seg = u % r.nseg, col = u / r.nseg;
    z0 = (col % r.nzc) * ring::ZT;
    bx = col / r.nzc;
    ys = (int)((long long)seg * r.a.Y / r.nseg);
    ye = (int)((long long)(seg + 1) * r.a.Y / r.nseg);
}

// accumulator block of virtual output row v: descending, so that the rows
// v + 2, v + 1, v fed by one input row are consecutive blocks
__device__ __forceinline__ uint32_t ring_blk(uint32_t v) { return (ring::NBLK - v % ring::NBLK) % ring::NBLK; }

// MMA q = 2 (3 dxi + dzi) + ks of an input row: descriptor offsets (16-byte
// units) of its A operand (from the slot's first run: z row 15 + dzi of run
// dxi, plus 32 bytes for the second K-step) and of its B operand (from the
// staged weights)
__host__ __device__ constexpr uint64_t ring_aoff(int q) {
    return (uint64_t)(((q >> 1) / 3) * (ring::RUN / 16) + (15 + (q >> 1) % 3) * 4 + 2 * (q & 1));
}
__host__ __device__ constexpr uint64_t ring_boff(int q) { return (uint64_t)(((q >> 1) * 12 * 4 + 2 * (q & 1)) * 8); }

__device__ __forceinline__ void tmem_st16_zero(uint32_t taddr) {
    const uint32_t z = 0;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(z)
        : "memory");
}

template <int EPI>
__global__ void __launch_bounds__(ring::NTH, 1)
    conv_ring_kernel(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap hmap, RingArgs r) {
    using namespace ring;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* sm = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);  // swizzle atoms: 1024-aligned
    unsigned char* swb = sm;
    unsigned char* sring = sm + WB;
    const uint32_t full = smem_addr(sm + BAR), tfull = full + 8 * NS, tempty = tfull + 8 * NBLK;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + BAR + 8 * (NS + 2 * NBLK));
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ConvArgs& a = r.a;
    const int X = a.X, Y = a.Y, Z = a.Z;

    // weights [t][co][ci] -> [dx][dz][n = 32 (dy+1) + co][ci]: one input row feeds the output rows
    // y' + 1 (dy = -1), y' (dy = 0), y' - 1 (dy = +1) through N = 96 stacked columns
    for (int e = threadIdx.x; e < 9 * 96 * 4; e += NTH) {
        const int kg = e & 3, n = (e >> 2) % 96, dd = e / (96 * 4), dxi = dd / 3, dzi = dd % 3;
        const int t = 9 * dxi + 3 * (n >> 5) + dzi, co = n & 31;
        const uint4 v = *reinterpret_cast<const uint4*>(a.w + (t * 32 + co) * 32 + kg * 8);
        *reinterpret_cast<uint4*>(swb + (((dd * 12 + (n >> 3)) * 4 + kg) * 8 + (n & 7)) * 16) = v;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "n"(NBLK * 32)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(full + 8 * s, 1);
        for (int c = 0; c < NBLK; ++c) {
            mbar_init(tfull + 8 * c, 1);
            mbar_init(tempty + 8 * c, NEPI);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // staged weights -> MMA operand reads
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    if (warp >= 2) {  // every accumulator block starts at zero; the MMAs only accumulate
        const uint32_t tq = tmem + ((uint32_t)((warp & 3) * 32) << 16) + ((warp - 2) >> 2) * 16;
        for (int c = 0; c < NBLK; ++c) tmem_st16_zero(tq + c * 32);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        // A slot is refilled once the MMAs of the row it last held have completed:
        // the MMA warp's commit on that row's accumulator block (virtual row
        // vslot[slot]) already signals it, so the slot needs no barrier of its own.
        uint32_t k = 0, V = 0;  // slots issued; first virtual row of the unit
        uint32_t vslot[NS];
        bool ok = true;
        for (int u = blockIdx.x; u < r.nunits && ok; u += gridDim.x) {
            int bx, z0, ys, ye;
            ring_unit(r, u, bx, z0, ys, ye);
            const int b = bx / X, x = bx - b * X;
            for (int j = -1; j <= ye - ys; ++j) {
                const int yp = (ys + j + Y) % Y;
                const uint32_t slot = k % NS;
                uint32_t w_ok = 1;
                if (lane == 0 && k >= NS)
                    w_ok = ring_wait(tfull + 8 * ring_blk(vslot[slot]), (vslot[slot] / NBLK) & 1, abort_flag);
                vslot[slot] = V + (uint32_t)(j + 1);
                if (!__shfl_sync(0xffffffffu, w_ok, 0)) {
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    const uint32_t base = smem_addr(sring + slot * SLOT);
                    const int zl = (z0 - 16 + Z) % Z, zr = (z0 + ZT) % Z;  // periodic z halo: 16-row boxes
                    mbar_expect_tx(full + 8 * slot, SLOT_TX);
#pragma unroll
                    for (int dxi = 0; dxi < 3; ++dxi) {
                        const int bxx = b * X + (x + dxi - 1 + X) % X;
                        const uint32_t run = base + dxi * RUN;
                        tma_load4(run + 16 * 64, &map, 0, z0, yp, bxx, full + 8 * slot);
                        tma_load4(run, &hmap, 0, zl, yp, bxx, full + 8 * slot);
                        tma_load4(run + (16 + ZT) * 64, &hmap, 0, zr, yp, bxx, full + 8 * slot);
                    }
                }
                __syncwarp();
                ++k;
            }
            V += (uint32_t)(ye - ys) + 4;
        }
        if (!ok && lane == 0)  // let this CTA's copies in flight land before it exits (bounded)
            for (uint32_t q = (k > (uint32_t)NS ? k - NS : 0); q < k; ++q) tc_wait(full + 8 * (q % NS), (q / NS) & 1);
    } else if (warp == 1) {
        // ------------------------------------------------------- MMA issuer
        // The whole warp walks the schedule (descriptors stay warp-uniform);
        // lane 0 waits, issues and commits. Input row i of a unit (y' = ys-1+i)
        // feeds virtual rows V+i+2, V+i+1, V+i (output rows y'+1, y', y'-1);
        // virtual rows V .. V+L+3 hold output rows ys-2 .. ye+1, of which the
        // first and last two are partial and discarded.
        constexpr uint32_t I96 = idesc_bf16(ZT, 96), I64 = idesc_bf16(ZT, 64), I32 = idesc_bf16(ZT, 32);
        const uint32_t ring0 = smem_addr(sring);
        const uint64_t bdesc0 = sdesc(smem_addr(swb), 128, 512);
        uint32_t k = 0, V = 0, last_v = 0;
        uint32_t vready = NBLK - 1;  // virtual rows <= vready have a free (zeroed) accumulator block
        bool ok = true, issued = false;
        for (int u = blockIdx.x; u < r.nunits && ok; u += gridDim.x) {
            int bx, z0, ys, ye;
            ring_unit(r, u, bx, z0, ys, ye);
            const uint32_t L = (uint32_t)(ye - ys);
            for (uint32_t i = 0; i <= L + 1; ++i, ++k) {
                // blocks are claimed 8 rows at a time (rows up to V+i+9, freed by the epilogue
                // once it has read rows up to V+i-7), so the tensor-memory fence that orders
                // the epilogue's reads before these MMAs runs once per 8 input rows. Every
                // epilogue warp frees rows in order, so the phase of the last claimed block
                // (row V+i-7 freed by all warps) implies the earlier ones: one probe, not 8,
                // of a barrier the tensor core's operand reads make slow to reach.
                const bool claim = V + i + 2 > vready;
                uint32_t w_ok = 1;
                if (lane == 0) {
                    const uint32_t vc = V + i + 9;
                    if (claim) w_ok = ring_wait(tempty + 8 * ring_blk(vc), ((vc / NBLK) & 1) ^ 1, abort_flag);
                    if (w_ok) w_ok = ring_wait(full + 8 * (k % NS), (k / NS) & 1, abort_flag);
                }
                if (!__shfl_sync(0xffffffffu, w_ok, 0)) {
                    ok = false;
                    break;
                }
                if (claim) {
                    vready = V + i + 9;
                    fence_after();
                }
                const uint64_t adesc = sdesc_sw64(ring0 + (k % NS) * SLOT);
                const uint32_t b0 = ring_blk(V + i + 2);  // blocks b0, b0+1, b0+2 (mod 16)
                // 18 MMAs (dx, dz, ks); where the three blocks wrap past the last
                // column, each splits into two. One (warp-uniform) branch per input
                // row keeps the unrolled issue sequences free of per-MMA control
                // flow; the warp stays converged and lane 0 issues (and commits).
                {
                    if (b0 <= NBLK - 3) {
#pragma unroll
                        for (int q = 0; q < 18; ++q)
                            tc_mma_lane0(tmem + b0 * 32, adesc + ring_aoff(q), bdesc0 + ring_boff(q), I96);
                    } else if (b0 == NBLK - 2) {
#pragma unroll
                        for (int q = 0; q < 18; ++q) {
                            tc_mma_lane0(tmem + b0 * 32, adesc + ring_aoff(q), bdesc0 + ring_boff(q), I64);
                            tc_mma_lane0(tmem, adesc + ring_aoff(q), bdesc0 + ring_boff(q) + 8 * 4 * 8, I32);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 18; ++q) {
                            tc_mma_lane0(tmem + b0 * 32, adesc + ring_aoff(q), bdesc0 + ring_boff(q), I32);
                            tc_mma_lane0(tmem, adesc + ring_aoff(q), bdesc0 + ring_boff(q) + 4 * 4 * 8, I64);
                        }
                    }
                }
                if (lane == 0) {
                    tc_commit(tfull + 8 * ring_blk(V + i));  // virtual row V+i has all its inputs; slot k is free
                    if (i == L + 1) {
                        tc_commit(tfull + 8 * ring_blk(V + L + 2));
                        tc_commit(tfull + 8 * ring_blk(V + L + 3));
                    }
                }
                issued = true;
                last_v = V + i;
                __syncwarp();
            }
            V += L + 4;
        }
        if (!ok && lane == 0 && issued)  // let the last MMAs land before the accumulators are freed (bounded)
            tc_wait(tfull + 8 * ring_blk(last_v), (last_v / NBLK) & 1);
        __syncwarp();
    } else {
        // --------------------------------------------------------- epilogue
        const int q4 = warp & 3, h = (warp - 2) >> 2;  // accumulator lanes 32 q4 .., columns 16 h ..
        float* stg = reinterpret_cast<float*>(sm + STG + (warp - 2) * STG_WARP);
        float bias[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) bias[i] = a.bias ? a.bias[h * 16 + i] : 0.f;
        uint32_t v = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < r.nunits && ok; u += gridDim.x) {
            int bx, z0, ys, ye;
            ring_unit(r, u, bx, z0, ys, ye);
            const int L = ye - ys;
            for (int jv = 0; jv < L + 4; ++jv, ++v) {
                const uint32_t blk = ring_blk(v);
                uint32_t w_ok = 1;
                if (lane == 0) w_ok = ring_wait(tfull + 8 * blk, (v / NBLK) & 1, abort_flag);
                if (!__shfl_sync(0xffffffffu, w_ok, 0)) {
                    ok = false;
                    break;
                }
                fence_after();
                uint32_t acc[16];
                const uint32_t tq = tmem + ((uint32_t)(q4 * 32) << 16) + blk * 32 + h * 16;
                tmem_ld16(tq, acc);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                tmem_st16_zero(tq);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty + 8 * blk);
                if (jv >= 2 && jv < L + 2) {
                    const long long vox0 = ((long long)bx * Y + (ys + jv - 2)) * Z + z0 + q4 * 32;
                    if (EPI == EVX_NN_EPI_RESID32)
                        resid32_staged(a, vox0, h * 16, acc, bias, stg, lane);
                    else
                        epilogue_store<EPI, 16>(a, vox0 + lane, h * 16, acc, bias);
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(NBLK * 32) : "memory");
}

// ---------------------------------------------------- unpipelined tile kernel
// Implicit GEMM on the 5th-generation tensor cores: per tile of 128 output
// voxels (2 rows x 64 z) D[128 x 32] (FP32, tensor memory) accumulates
// 27 taps x 2 K-steps of A[128 x 16] (BF16 activations) times B[16 x 32]
// (BF16 weights). Operands sit in shared memory in the no-swizzle K-major
// core-matrix layout (8 rows x 16 bytes per 128-byte core matrix): weights as
// [t][co/8][ci/8][8][8], the halo as three copies shifted by dz = -1, 0, +1 so
// that every tap's A operand starts on an 8-voxel boundary:
// [dz][halo row][v/8][ci/8][8][8]. Core matrices adjacent along K are 128 B
// apart (leading byte offset), along M/N 512 B (stride byte offset).
// One thread issues the MMAs, the commit arrives on an mbarrier (bounded
// wait), and each of the 4 warps reads its 32 accumulator lanes (one voxel
// row each) with tcgen05.ld for the fused epilogue.
template <int EPI>
__global__ void __launch_bounds__(128, 1) conv_tc_kernel(ConvArgs a) {
    constexpr int C = 32, HALO = HR * 8 * 4 * 128;  // bytes per dz copy
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* swb = smem_raw;                          // weights: 27 * 4 * 4 * 128 B
    unsigned char* shalo = smem_raw + 27 * 4 * 4 * 128;     // 3 copies of HALO bytes
    uint64_t* bar = reinterpret_cast<uint64_t*>(shalo + 3 * HALO);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // weights -> core-matrix layout
    for (int e = threadIdx.x; e < 27 * C * 4; e += 128) {  // 16-byte pieces: (t, co, cig)
        const int cig = e & 3, co = (e >> 2) % C, t = e / (4 * C);
        const uint4 v = *reinterpret_cast<const uint4*>(a.w + ((long long)t * C + co) * C + cig * 8);
        *reinterpret_cast<uint4*>(swb + (((t * 4 + (co >> 3)) * 4 + cig) * 8 + (co & 7)) * 16) = v;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_addr(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    float bias[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) bias[i] = a.bias ? a.bias[i] : 0.f;
    constexpr uint32_t IDESC = idesc_bf16(128, 32);
    uint32_t parity = 0;
    bool failed = false;
    for (int tile = blockIdx.x; tile < a.ntiles && !failed; tile += gridDim.x) {
        int b, x, y0, z0;
        tile_coords(tile, a.X, a.Y, a.Z, b, x, y0, z0);
        // halo -> three dz-shifted copies in core-matrix layout
        for (int e = threadIdx.x; e < HR * (TZ + 2) * 4; e += 128) {
            const int cig = e & 3, rem = e >> 2, zi = rem % (TZ + 2), nb = rem / (TZ + 2);
            const int dx = nb / (TY + 2) - 1, yi = nb % (TY + 2) - 1;
            const int xx = (x + dx + a.X) % a.X, yy = (y0 + yi + a.Y) % a.Y, zz = (z0 + zi - 1 + a.Z) % a.Z;
            const long long vox = (((long long)b * a.X + xx) * a.Y + yy) * a.Z + zz;
            const uint4 v = *reinterpret_cast<const uint4*>(a.in + vox * C + cig * 8);
#pragma unroll
            for (int s = 0; s < 3; ++s) {  // copy s holds position p = zi - s (dz = s - 1)
                const int p = zi - s;
                if (p >= 0 && p < TZ)
                    *reinterpret_cast<uint4*>(shalo + s * HALO + (((nb * 8 + (p >> 3)) * 4 + cig) * 8 + (p & 7)) * 16) =
                        v;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (threadIdx.x == 0) {
            const uint32_t hbase = smem_addr(shalo), wbase = smem_addr(swb);
            int k = 0;
            for (int t = 0; t < 27; ++t) {
                const int dxi = t / 9, dyi = (t / 3) % 3, s = t % 3;
                const int nb0 = dxi * (TY + 2) + dyi;  // halo row of the first output row (yl = 0)
#pragma unroll
                for (int ks = 0; ks < 2; ++ks, ++k) {
                    const uint64_t ad = sdesc(hbase + s * HALO + ((nb0 * 8) * 4 + 2 * ks) * 128, 128, 512);
                    const uint64_t bd = sdesc(wbase + (t * 16 + 2 * ks) * 128, 128, 512);
                    tc_mma(tmem, ad, bd, IDESC, k > 0);
                }
            }
            tc_commit(smem_addr(bar));
        }
        const bool ok = tc_wait(smem_addr(bar), parity);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        parity ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: thread = accumulator lane = voxel m of the tile (m < 64: row y0, else y0 + 1)
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int m = warp * 32 + lane;
        const long long vox = (((long long)b * a.X + x) * a.Y + y0 + (m >> 6)) * a.Z + z0 + (m & 63);
        epilogue_store<EPI, 32>(a, vox, 0, r, bias);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // accumulator read before the next tile's MMAs overwrite it
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (failed && threadIdx.x == 0) {
        atomicExch(&g_tc_timeout, 1);
        tc_wait(smem_addr(bar), parity);  // let the outstanding commit land (bounded) before freeing TMEM
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}


}  // namespace evxnn

// =================================================================== host
namespace {
using namespace evxnn;

PFN_cuTensorMapEncodeTiled_v12000 nn_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
        else
            cudaGetLastError();
    }
    return fn;
}

// activations [B X][Y][Z][32] as a 4D BF16 tensor (32 channels, Z, Y, B X), box 32 channels x zrows z,
// written to shared memory in the 64-byte swizzle layout
bool ring_map(CUtensorMap* m, const ConvArgs& a, int zrows) {
    auto fn = nn_encode_fn();
    if (!fn || ((uintptr_t)a.in & 15)) return false;
    const cuuint64_t dims[4] = {32, (cuuint64_t)a.Z, (cuuint64_t)a.Y, (cuuint64_t)a.B * a.X};
    const cuuint64_t strides[3] = {64, (cuuint64_t)a.Z * 64, (cuuint64_t)a.Y * a.Z * 64};
    const cuuint32_t box[4] = {32, (cuuint32_t)zrows, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(a.in), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int EPI>
cudaError_t launch_ring(const ConvArgs& a, cudaStream_t st, int sms, bool* launched) {
    *launched = false;
    CUtensorMap map, hmap;
    if (a.Z % ring::ZT || !ring_map(&map, a, ring::ZT) || !ring_map(&hmap, a, 16)) return cudaSuccess;
    RingArgs r{};
    r.a = a;
    r.nzc = a.Z / ring::ZT;
    const long long ncol = (long long)a.B * a.X * r.nzc;
    int nseg = 1;  // split columns along y until there are enough units for an even spread
    while (ncol * nseg < 8LL * sms && nseg * 2 <= a.Y / 8) nseg *= 2;
    if (ncol * nseg > (1LL << 30)) return cudaSuccess;  // unit index would overflow int: not launched, tile kernel
    r.nseg = nseg;
    r.nunits = (int)(ncol * nseg);
    cudaError_t e = cudaFuncSetAttribute(conv_ring_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, ring::SMEM);
    if (e != cudaSuccess) return e;
    conv_ring_kernel<EPI><<<std::min(r.nunits, sms), ring::NTH, ring::SMEM, st>>>(map, hmap, r);
    *launched = true;
    return cudaGetLastError();
}

template <int EPI>
cudaError_t launch_tile(const ConvArgs& a0, cudaStream_t st, int sms) {
    ConvArgs a = a0;
    a.ntiles = a.B * a.X * (a.Y / TY) * (a.Z / TZ);
    const size_t smem = 27 * 4 * 4 * 128 + 3 * (size_t)HR * 8 * 4 * 128 + 16;
    cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    conv_tc_kernel<EPI><<<std::min(a.ntiles, sms), 128, smem, st>>>(a);
    return cudaGetLastError();
}

template <int EPI>
cudaError_t conv32_tc_epi(const ConvArgs& a, cudaStream_t st, int sms) {
    bool launched = false;
    const cudaError_t e = launch_ring<EPI>(a, st, sms, &launched);
    if (launched || e != cudaSuccess) return e;
    return launch_tile<EPI>(a, st, sms);
}
}  // namespace

namespace evxnn {

cudaError_t conv32_tc(const ConvArgs& a, int epilogue, cudaStream_t st, int sms) {
    switch (epilogue) {
        case EVX_NN_EPI_PLAIN: return conv32_tc_epi<EVX_NN_EPI_PLAIN>(a, st, sms);
        case EVX_NN_EPI_GELU: return conv32_tc_epi<EVX_NN_EPI_GELU>(a, st, sms);
        case EVX_NN_EPI_RESID: return conv32_tc_epi<EVX_NN_EPI_RESID>(a, st, sms);
        case EVX_NN_EPI_GELU_BWD: return conv32_tc_epi<EVX_NN_EPI_GELU_BWD>(a, st, sms);
        case EVX_NN_EPI_RESID32: return conv32_tc_epi<EVX_NN_EPI_RESID32>(a, st, sms);
    }
    return cudaErrorInvalidValue;
}

cudaError_t tc_take_timeout(int* flag) {
    cudaError_t e = cudaMemcpyFromSymbol(flag, g_tc_timeout, sizeof(int));
    if (e != cudaSuccess || !*flag) return e;
    const int zero = 0;
    return cudaMemcpyToSymbol(g_tc_timeout, &zero, sizeof(int));
}

}  // namespace evxnn
