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

struct __align__(16) CtrSmem {
    uint32_t te[256 * 32]; // table 0, one copy per lane
    uint4 rk[11];          // round keys, one 16-byte load per round
    uint4 rk_last_le;      // last round key with its bytes in stream order
};

// byte k of v, zero-extended
__device__ __forceinline__ uint32_t byte_of(uint32_t v, uint32_t k) { return __byte_perm(v, 0u, 0x4440u | k); }

// entry x of table 0 (lane-replicated: word 32 x + lane, so one multiply-add
// gives the address)
__device__ __forceinline__ uint32_t t0(const uint32_t *tel, uint32_t x) { return tel[x << 5]; }

// rotations by whole bytes: tables 1..3 from table 0
__device__ __forceinline__ uint32_t ror8(uint32_t v) { return __byte_perm(v, v, 0x0321); }
__device__ __forceinline__ uint32_t ror16(uint32_t v) { return __byte_perm(v, v, 0x1032); }
__device__ __forceinline__ uint32_t ror24(uint32_t v) { return __byte_perm(v, v, 0x2103); }

// one AES-128 block (FIPS-197 cipher, 32-bit table form) of the counter
// block nonce || blk; the keystream words come back with their bytes in
// stream order (ks[0] byte 0 is keystream byte 0), ready to XOR with
// little-endian loads
__device__ __forceinline__ void ctr_block(const CtrSmem &m, uint32_t lane, uint64_t nonce,
                                          uint64_t blk, uint32_t ks[4])
{
    const uint32_t *tel = m.te + lane;
    const uint4 k0 = m.rk[0];
    uint32_t s0 = (uint32_t)(nonce >> 32) ^ k0.x;
    uint32_t s1 = (uint32_t)nonce ^ k0.y;
    uint32_t s2 = (uint32_t)(blk >> 32) ^ k0.z;
    uint32_t s3 = (uint32_t)blk ^ k0.w;
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        const uint4 k = m.rk[r];
        const uint32_t n0 = t0(tel, byte_of(s0, 3)) ^ ror8(t0(tel, byte_of(s1, 2))) ^
                            ror16(t0(tel, byte_of(s2, 1))) ^ ror24(t0(tel, byte_of(s3, 0))) ^ k.x;
        const uint32_t n1 = t0(tel, byte_of(s1, 3)) ^ ror8(t0(tel, byte_of(s2, 2))) ^
                            ror16(t0(tel, byte_of(s3, 1))) ^ ror24(t0(tel, byte_of(s0, 0))) ^ k.y;
        const uint32_t n2 = t0(tel, byte_of(s2, 3)) ^ ror8(t0(tel, byte_of(s3, 2))) ^
                            ror16(t0(tel, byte_of(s0, 1))) ^ ror24(t0(tel, byte_of(s1, 0))) ^ k.z;
        const uint32_t n3 = t0(tel, byte_of(s3, 3)) ^ ror8(t0(tel, byte_of(s0, 2))) ^
                            ror16(t0(tel, byte_of(s1, 1))) ^ ror24(t0(tel, byte_of(s2, 0))) ^ k.w;
        s0 = n0;
        s1 = n1;
        s2 = n2;
        s3 = n3;
    }
    // last round: SubBytes, ShiftRows, AddRoundKey.  S[x] is byte 1 (and 2)
    // of table-0 entry x; the output bytes go straight to stream order.
    auto sub4 = [&](uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
        const uint32_t lo = __byte_perm(t0(tel, byte_of(a, 3)), t0(tel, byte_of(b, 2)), 0x0051);
        const uint32_t hi = __byte_perm(t0(tel, byte_of(c, 1)), t0(tel, byte_of(d, 0)), 0x0051);
        return __byte_perm(lo, hi, 0x5410);
    };
    const uint4 kl = m.rk_last_le;
    ks[0] = sub4(s0, s1, s2, s3) ^ kl.x;
    ks[1] = sub4(s1, s2, s3, s0) ^ kl.y;
    ks[2] = sub4(s2, s3, s0, s1) ^ kl.z;
    ks[3] = sub4(s3, s0, s1, s2) ^ kl.w;
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
    for (int i = threadIdx.x; i < 44; i += blockDim.x) {
        const uint32_t k = w.round_keys[i];
        (&m.rk[0].x)[i] = k;
        if (i >= 40)
            (&m.rk_last_le.x)[i - 40] = __byte_perm(k, 0, 0x0123);
    }
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
                uint4 r;
                r.x = t.x ^ ks[0];
                r.y = t.y ^ ks[1];
                r.z = t.z ^ ks[2];
                r.w = t.w ^ ks[3];
                *reinterpret_cast<uint4 *>(ch.out + o) = r;
            } else {
                for (int k = 0; k < 16 && o + (uint64_t)k < ch.bytes; ++k)
                    ch.out[o + k] = (uint8_t)(__ldcg(ch.in + o + k) ^ (uint8_t)(ks[k >> 2] >> (8 * (k & 3))));
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
