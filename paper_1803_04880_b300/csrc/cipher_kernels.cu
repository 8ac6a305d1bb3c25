// cipher_kernels.cu -- AES-128-CTR over large private fragments in a launch
// of its own.
//
// With one or two levels the private fragment (LL_L as int16) is half or an
// eighth of the input, and the cipher, not the transform, bounds the time.
// This kernel keeps one AES table in shared memory replicated once per lane
// (entry x of lane t at word 32 x + t), so the 32 lookups of a warp always
// fall in 32 different banks; the other three tables of the 32-bit table
// form are byte rotations of the first (FIPS-197 Sec. 5.1 combined into
// table lookups), and the last round's S-box is a byte of the same entry.
// The counter block is nonce (8 bytes big-endian) || block index (8 bytes
// big-endian); out = in XOR keystream, in may equal out.  The keystream does
// not depend on the data, so the kernel is launched as a programmatic
// dependent of the kernel before it: it builds its table and its first
// keystream blocks while that kernel still runs, and waits for it only
// before reading the fragment.  Buffers with three
// or more levels keep their cipher units inside the dependency-ordered
// launch, where the fragment is small.
#include "frag_internal.cuh"

namespace frag {

constexpr int kCtrThreads = 256;

struct CtrSmem {
    uint32_t te[256 * 32]; // table 0, one copy per lane
    uint32_t rk[44];
};

__device__ __forceinline__ uint32_t ror(uint32_t v, int s) { return __funnelshift_r(v, v, s); }

// one AES-128 block (FIPS-197 cipher): counter nonce || blk, keystream words
// in big-endian order
__device__ __forceinline__ void ctr_block(const CtrSmem &m, uint32_t lane, uint64_t nonce,
                                          uint64_t blk, uint32_t ks[4])
{
    const uint32_t *te = m.te + lane;
    uint32_t s0 = (uint32_t)(nonce >> 32) ^ m.rk[0];
    uint32_t s1 = (uint32_t)nonce ^ m.rk[1];
    uint32_t s2 = (uint32_t)(blk >> 32) ^ m.rk[2];
    uint32_t s3 = (uint32_t)blk ^ m.rk[3];
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        const uint32_t t0 = te[(s0 >> 24) << 5] ^ ror(te[((s1 >> 16) & 255) << 5], 8) ^
                            ror(te[((s2 >> 8) & 255) << 5], 16) ^ ror(te[(s3 & 255) << 5], 24) ^
                            m.rk[4 * r];
        const uint32_t t1 = te[(s1 >> 24) << 5] ^ ror(te[((s2 >> 16) & 255) << 5], 8) ^
                            ror(te[((s3 >> 8) & 255) << 5], 16) ^ ror(te[(s0 & 255) << 5], 24) ^
                            m.rk[4 * r + 1];
        const uint32_t t2 = te[(s2 >> 24) << 5] ^ ror(te[((s3 >> 16) & 255) << 5], 8) ^
                            ror(te[((s0 >> 8) & 255) << 5], 16) ^ ror(te[(s1 & 255) << 5], 24) ^
                            m.rk[4 * r + 2];
        const uint32_t t3 = te[(s3 >> 24) << 5] ^ ror(te[((s0 >> 16) & 255) << 5], 8) ^
                            ror(te[((s1 >> 8) & 255) << 5], 16) ^ ror(te[(s2 & 255) << 5], 24) ^
                            m.rk[4 * r + 3];
        s0 = t0;
        s1 = t1;
        s2 = t2;
        s3 = t3;
    }
    // last round: SubBytes, ShiftRows, AddRoundKey; S[x] is byte 2 of table 0
    auto sb = [&](uint32_t x) { return (te[x << 5] >> 16) & 255u; };
    ks[0] = ((sb(s0 >> 24) << 24) | (sb((s1 >> 16) & 255) << 16) | (sb((s2 >> 8) & 255) << 8) |
             sb(s3 & 255)) ^ m.rk[40];
    ks[1] = ((sb(s1 >> 24) << 24) | (sb((s2 >> 16) & 255) << 16) | (sb((s3 >> 8) & 255) << 8) |
             sb(s0 & 255)) ^ m.rk[41];
    ks[2] = ((sb(s2 >> 24) << 24) | (sb((s3 >> 16) & 255) << 16) | (sb((s0 >> 8) & 255) << 8) |
             sb(s1 & 255)) ^ m.rk[42];
    ks[3] = ((sb(s3 >> 24) << 24) | (sb((s0 >> 16) & 255) << 16) | (sb((s1 >> 8) & 255) << 8) |
             sb(s2 & 255)) ^ m.rk[43];
}

__global__ void __launch_bounds__(kCtrThreads) ctr_kernel(CtrWork w)
{
    extern __shared__ __align__(16) uint8_t smem[];
    CtrSmem &m = *reinterpret_cast<CtrSmem *>(smem);
    grid_release();
    // table 0 into shared memory, one copy per lane: each warp takes 32
    // entries with one coalesced load and writes entry x as 32 consecutive
    // words (x, lane), conflict-free
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t base = (threadIdx.x >> 5) * 32; base < 256; base += (blockDim.x >> 5) * 32) {
        const uint32_t v = __ldg(w.aes_tables + base + lane);
#pragma unroll 8
        for (int k = 0; k < 32; ++k)
            m.te[(base + k) * 32 + lane] = __shfl_sync(0xffffffffu, v, k);
    }
    for (int i = threadIdx.x; i < 44; i += blockDim.x)
        m.rk[i] = w.round_keys[i];
    __syncthreads();
    const uint64_t nchunks = w.chunks ? w.nchunks
                                      : (w.single.nblocks + w.single_chunk - 1) / w.single_chunk;
    for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        CtrChunk ch;
        if (w.chunks) {
            ch = w.chunks[c];
        } else {
            ch = w.single;
            ch.first_block = c * w.single_chunk;
            ch.nblocks = min(w.single_chunk, w.single.nblocks - ch.first_block);
        }
        const bool vec = (((uintptr_t)ch.in | (uintptr_t)ch.out) & 15u) == 0;
        for (uint64_t i = threadIdx.x; i < ch.nblocks; i += blockDim.x) {
            const uint64_t b = ch.first_block + i;
            uint32_t ks[4];
            ctr_block(m, lane, ch.nonce, b, ks);
            grid_wait(); // the fragment is complete from here on (returns at once after the first)
            const uint64_t o = 16 * b;
            if (vec && o + 16 <= ch.bytes) {
                // L2-coherent load: the kernel before this one wrote the
                // fragment while this grid was already resident, so the
                // read-only (non-coherent) path is not allowed here
                const uint4 t = __ldcg(reinterpret_cast<const uint4 *>(ch.in + o));
                uint4 r; // keystream bytes in stream order = big-endian words
                r.x = t.x ^ __byte_perm(ks[0], 0, 0x0123);
                r.y = t.y ^ __byte_perm(ks[1], 0, 0x0123);
                r.z = t.z ^ __byte_perm(ks[2], 0, 0x0123);
                r.w = t.w ^ __byte_perm(ks[3], 0, 0x0123);
                *reinterpret_cast<uint4 *>(ch.out + o) = r;
            } else {
                for (int k = 0; k < 16 && o + (uint64_t)k < ch.bytes; ++k)
                    ch.out[o + k] = (uint8_t)(__ldcg(ch.in + o + k) ^ (uint8_t)(ks[k >> 2] >> (24 - 8 * (k & 3))));
            }
        }
    }
}

static cudaError_t ctr_attr()
{
    return cudaFuncSetAttribute((const void *)ctr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(CtrSmem));
}

cudaError_t launch_ctr(const CtrWork &w, uint32_t grid, cudaStream_t stream)
{
    cudaError_t e = ctr_attr();
    if (e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kCtrThreads);
    cfg.dynamicSmemBytes = sizeof(CtrSmem);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, ctr_kernel, w);
}

cudaError_t ctr_occupancy(int *blocks_per_sm)
{
    cudaError_t e = ctr_attr();
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void *)ctr_kernel,
                                                         kCtrThreads, sizeof(CtrSmem));
}

} // namespace frag
