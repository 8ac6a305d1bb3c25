// cipher_kernels.cu -- AES-128-CTR over private fragments in a launch of
// their own (Sec. 5.2.1: the private fragment is encrypted with AES; CTR as
// in SP 800-38A).
//
// Buffers whose levels the fused kernel does not finish, the block mode, the
// packed fragments and the full-buffer comparator encipher here.  The kernel
// uses the two-table AES of aes_tt.cuh: T0 and T2 once per lane in 64 KB of
// shared memory placed on a 64 KB boundary of the shared window, so every
// lookup is one byte permute and one shared load, and a round column one
// rotation.  One block of 1024 threads an SM; work goes by warps: a warp
// takes a turn of a fragment (a fragment of the launch's list, found by
// binary search over the turns, or a slice of a lone fragment) and its lanes
// take every 32nd block of it.  The round-1
// constants of the chunk's nonce are computed once per chunk (only the
// low block word varies within it).  The counter block is nonce (8 bytes
// big-endian) || block index (8 bytes big-endian); out = in XOR keystream,
// in may equal out.  Launched as a programmatic dependent of the kernel
// before it: the table is built while that kernel drains, and the fragment
// is read only after griddepcontrol.wait.
#include "aes_tt.cuh"

namespace frag {

// dynamic shared memory: enough to place the 64 KB table on a 64 KB window
// boundary wherever the dynamic part starts, from 0 up to 64 KB
constexpr size_t kCtrSmem = 2 * aes::kDualBytes;

__global__ void __launch_bounds__(kCtrThreads, 1) ctr_kernel(CtrWork w)
{
    extern __shared__ __align__(16) uint8_t smem[];
    grid_release();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t tab = aes::dual_table_at((uint32_t)__cvta_generic_to_shared(smem));
    aes::build_dual<kCtrThreads>(tab, w.aes_tables);
    __syncthreads();
    const aes::Lut L = aes::make_lut(tab, lane);
    grid_wait(); // the fragment is complete from here on
    const uint64_t nturns = w.frags ? w.nturns : (w.single.nblocks + w.turn_blocks - 1) / w.turn_blocks;
    // turn c of the launch goes to warp c / grid of CTA c % grid, so a launch
    // of few turns still spreads them over every CTA (every SM)
    const uint64_t warps = (uint64_t)gridDim.x * (kCtrThreads / 32);
    for (uint64_t c = (uint64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x; c < nturns; c += warps) {
        CtrChunk ch;
        uint64_t first;
        if (w.frags) { // the fragment whose turns hold c
            uint64_t lo = 0, hi = w.nfrags;
            while (hi - lo > 1) {
                const uint64_t mid = (lo + hi) >> 1;
                if (__ldg(w.turn_start + mid) <= c)
                    lo = mid;
                else
                    hi = mid;
            }
            ch = w.frags[lo];
            first = (c - __ldg(w.turn_start + lo)) * w.turn_blocks;
        } else {
            ch = w.single;
            first = c * w.turn_blocks;
        }
        ch.nblocks = min(w.turn_blocks, ch.nblocks - first);
        ch.first_block += first;
        const bool vec = (((uintptr_t)ch.in | (uintptr_t)ch.out) & 15u) == 0;
        aes::Round1 R = aes::round1_consts(L, w.keys, ch.nonce, (uint32_t)(ch.first_block >> 32));
        for (uint64_t i = lane; i < ch.nblocks; i += 32) {
            const uint64_t b = ch.first_block + i;
            if ((uint32_t)(b >> 32) != R.hi) // a 2^32-block boundary (fragments of 64 GiB)
                R = aes::round1_consts(L, w.keys, ch.nonce, (uint32_t)(b >> 32));
            const uint64_t o = 16 * b;
            const bool whole = vec && o + 16 <= ch.bytes;
            // L2-coherent load, issued before the rounds: the kernel before
            // this one wrote the fragment while this grid was already
            // resident, so the read-only (non-coherent) path is not allowed
            uint4 t = make_uint4(0, 0, 0, 0);
            if (whole)
                t = __ldcg(reinterpret_cast<const uint4 *>(ch.in + o));
            uint32_t ks[4];
            aes::ctr_block2(L, w.keys, R, (uint32_t)b, ks);
            if (whole) {
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
    static std::atomic<uint64_t> done{0};
    return smem_attr_once((const void *)ctr_kernel, (int)kCtrSmem, done);
}

cudaError_t launch_ctr(const CtrWork &w, uint32_t grid, cudaStream_t stream)
{
    cudaError_t e = ctr_attr();
    if (e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kCtrThreads);
    cfg.dynamicSmemBytes = kCtrSmem;
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
                                                         kCtrThreads, kCtrSmem);
}

} // namespace frag

// ---------------------------------------------------------------------------
// bitsliced AES-128-CTR (aes_bs.cuh): the measured alternative to the table
// form.  A warp takes a chunk of 1,024 counter blocks; lane l computes blocks
// base + 32 j + l (j = 0..31) as one bitsliced state, so its counter planes
// need no transpose (bits 0..4 of the block index are the lane's, bits 5..9
// the fixed patterns of j, the rest the chunk's), and after the last round
// four 32 x 32 transposes give each block's 16 keystream bytes, which the
// warp XORs into the data 512 contiguous bytes at a time.
// ---------------------------------------------------------------------------
#include "aes_bs.cuh"

namespace frag {

constexpr int kBsThreads = 128;

__global__ void __launch_bounds__(kBsThreads, 2) ctr_bs_kernel(const __grid_constant__ BsCtrWork w)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (kBsThreads / 32);
    const bool vec = (((uintptr_t)w.in | (uintptr_t)w.out) & 15u) == 0;
    const uint32_t jpat[5] = {0xaaaaaaaau, 0xccccccccu, 0xf0f0f0f0u, 0xff00ff00u, 0xffff0000u};
    for (uint64_t ch = (uint64_t)blockIdx.x * (kBsThreads / 32) + (threadIdx.x >> 5); ch < w.nchunks;
         ch += warps) {
        const uint64_t base = ch * (uint64_t)bs::kChunkBlocks;
        // the counter blocks nonce || (base + 32 j + lane), big-endian, with
        // round key 0
        uint32_t x[128];
#pragma unroll
        for (int p = 0; p < 16; ++p) {
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                uint32_t v;
                if (p < 8) {
                    v = 0u - (uint32_t)((w.nonce >> (8 * (7 - p) + b)) & 1u);
                } else {
                    const int q = 8 * (15 - p) + b; // bit q of the block index
                    if (q < 5)
                        v = 0u - ((lane >> q) & 1u);
                    else if (q < 10)
                        v = jpat[q - 5];
                    else
                        v = 0u - (uint32_t)((base >> q) & 1u);
                }
                x[8 * p + b] = v ^ w.w[0][8 * p + b];
            }
        }
#pragma unroll 1
        for (int r = 1; r < 10; ++r) {
            uint32_t y[128], z[128];
            bs::sub_shift(x, y);
            bs::mix(y, z);
#pragma unroll
            for (int k = 0; k < 128; ++k)
                x[k] = z[k] ^ w.w[r][k];
        }
        {
            uint32_t y[128];
            bs::sub_shift(x, y);
#pragma unroll
            for (int k = 0; k < 128; ++k)
                x[k] = y[k] ^ w.w[10][k];
        }
        // keystream word g of block j = bytes 4 g .. 4 g + 3 little-endian
        uint32_t T[4][32];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
#pragma unroll
            for (int k = 0; k < 32; ++k)
                T[g][k] = x[8 * (4 * g + k / 8) + k % 8];
            bs::transpose32(T[g]);
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const uint64_t o = 16 * (base + 32 * (uint64_t)j + lane);
            if (o >= w.bytes)
                continue;
            if (vec && o + 16 <= w.bytes) {
                const uint4 t = __ldcs(reinterpret_cast<const uint4 *>(w.in + o));
                __stcs(reinterpret_cast<uint4 *>(w.out + o),
                       make_uint4(t.x ^ T[0][j], t.y ^ T[1][j], t.z ^ T[2][j], t.w ^ T[3][j]));
            } else {
                for (int k = 0; k < 16 && o + k < w.bytes; ++k)
                    w.out[o + k] = (uint8_t)(w.in[o + k] ^ (uint8_t)(T[k >> 2][j] >> (8 * (k & 3))));
            }
        }
    }
}

cudaError_t launch_ctr_bs(const BsCtrWork &w, cudaStream_t stream)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)ctr_bs_kernel, kBsThreads, 0);
    if (e != cudaSuccess)
        return e;
    const uint64_t need = (w.nchunks + kBsThreads / 32 - 1) / (kBsThreads / 32);
    const uint64_t most = (uint64_t)sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
    const uint32_t grid = (uint32_t)(need < most ? need : most);
    ctr_bs_kernel<<<grid, kBsThreads, 0, stream>>>(w);
    return cudaGetLastError();
}

} // namespace frag
