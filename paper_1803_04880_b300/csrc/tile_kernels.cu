// tile_kernels.cu -- the persistent tile kernel of the allocation-free
// protect (LeGall 5/3 forward of 1 to 5 levels with AES-128-CTR on the final
// LL band), for sm_103a.
//
// Each CTA is persistent: it loads the AES tables and round keys into shared
// memory once, then takes tiles from a device work queue until none are
// left.  A tile owns a square of level-0 pixels of one buffer; the CTA stages
// the tile plus its lifting halo in shared memory and runs every level there
// (fast_tiles.cuh: Eq. 5.1 predict, Eq. 5.2 update, rows before columns
// within a level, Sec. 5.2.2), so the only device memory it touches besides
// the caller's buffers is the queue, the descriptors and the tables: no level
// scratch.  Input bytes inside the halo are read by both neighbouring tiles.
#include "frag_internal.cuh"

namespace frag {

struct AesSmem {
    uint32_t T[4][256]; // T[i][a] = MixColumns column of S[a], rotated right by 8i bits
    uint32_t S[256];    // S-box, one entry per word
    uint32_t rk[44];    // round keys, big-endian words
};

// AES-128 encryption of one counter block (FIPS-197 cipher in its 32-bit
// table form: SubBytes + ShiftRows + MixColumns per round as four lookups).
// Counter block = nonce || blk, both big-endian; words are big-endian columns.
__device__ __forceinline__ void aes_ctr_block(const AesSmem &a, uint64_t nonce, uint64_t blk,
                                              uint32_t ks[4])
{
    uint32_t s0 = (uint32_t)(nonce >> 32) ^ a.rk[0];
    uint32_t s1 = (uint32_t)nonce ^ a.rk[1];
    uint32_t s2 = (uint32_t)(blk >> 32) ^ a.rk[2];
    uint32_t s3 = (uint32_t)blk ^ a.rk[3];
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        const uint32_t t0 = a.T[0][s0 >> 24] ^ a.T[1][(s1 >> 16) & 255] ^
                            a.T[2][(s2 >> 8) & 255] ^ a.T[3][s3 & 255] ^ a.rk[4 * r];
        const uint32_t t1 = a.T[0][s1 >> 24] ^ a.T[1][(s2 >> 16) & 255] ^
                            a.T[2][(s3 >> 8) & 255] ^ a.T[3][s0 & 255] ^ a.rk[4 * r + 1];
        const uint32_t t2 = a.T[0][s2 >> 24] ^ a.T[1][(s3 >> 16) & 255] ^
                            a.T[2][(s0 >> 8) & 255] ^ a.T[3][s1 & 255] ^ a.rk[4 * r + 2];
        const uint32_t t3 = a.T[0][s3 >> 24] ^ a.T[1][(s0 >> 16) & 255] ^
                            a.T[2][(s1 >> 8) & 255] ^ a.T[3][s2 & 255] ^ a.rk[4 * r + 3];
        s0 = t0;
        s1 = t1;
        s2 = t2;
        s3 = t3;
    }
    ks[0] = ((a.S[s0 >> 24] << 24) | (a.S[(s1 >> 16) & 255] << 16) |
             (a.S[(s2 >> 8) & 255] << 8) | a.S[s3 & 255]) ^ a.rk[40];
    ks[1] = ((a.S[s1 >> 24] << 24) | (a.S[(s2 >> 16) & 255] << 16) |
             (a.S[(s3 >> 8) & 255] << 8) | a.S[s0 & 255]) ^ a.rk[41];
    ks[2] = ((a.S[s2 >> 24] << 24) | (a.S[(s3 >> 16) & 255] << 16) |
             (a.S[(s0 >> 8) & 255] << 8) | a.S[s1 & 255]) ^ a.rk[42];
    ks[3] = ((a.S[s3 >> 24] << 24) | (a.S[(s0 >> 16) & 255] << 16) |
             (a.S[(s1 >> 8) & 255] << 8) | a.S[s2 & 255]) ^ a.rk[43];
}

__device__ __forceinline__ uint32_t ks_byte(const uint32_t ks[4], int k)
{
    return (ks[k >> 2] >> (24 - 8 * (k & 3))) & 255u;
}

} // namespace frag

#include "fast_tiles.cuh"

namespace frag {

__device__ __forceinline__ void load_aes(AesSmem &a, const Work &w)
{
    uint32_t *dst = &a.T[0][0];
    for (int i = threadIdx.x; i < kAesWords; i += blockDim.x)
        dst[i] = w.aes_tables[i];
    for (int i = threadIdx.x; i < 44; i += blockDim.x)
        a.rk[i] = w.round_keys[i];
    __syncthreads();
}

// the job that owns global tile t (binary search over the tile prefix)
__device__ __forceinline__ const Job *find_job(const Work &w, uint64_t t, uint64_t &local)
{
    uint32_t lo = 0, hi = w.njobs; // tile_start[lo] <= t < tile_start[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        if (w.tile_start[mid] <= t)
            lo = mid;
        else
            hi = mid;
    }
    local = t - w.tile_start[lo];
    return &w.jobs[lo];
}

__global__ void __launch_bounds__(kThreads, 1) tile_kernel(Work w)
{
    extern __shared__ __align__(16) uint32_t smem[];
    AesSmem &aes = *reinterpret_cast<AesSmem *>(smem);
    uint32_t *S = smem + sizeof(AesSmem) / 4;
    __shared__ unsigned long long s_tile;
    load_aes(aes, w);

    for (;;) {
        if (threadIdx.x == 0)
            s_tile = atomicAdd(w.queue, 1ull);
        __syncthreads();
        const uint64_t t = s_tile;
        __syncthreads();
        if (t >= w.total_tiles)
            break;
        uint64_t local;
        const Job j = *find_job(w, t, local);
        // a descriptor that does not match its own tile count, level count
        // or tile side: record it (code 2) and stop this CTA
        if (j.tiles_x == 0 || local >= (uint64_t)j.tiles_x * j.tiles_y || j.L < 1 ||
            j.L > kTileMaxLevels || j.tile != tile_side(j.L)) {
            if (threadIdx.x == 0)
                atomicCAS(w.err, 0, 2);
            break;
        }
        const uint32_t tx = (uint32_t)(local % j.tiles_x), ty = (uint32_t)(local / j.tiles_x);
        switch (j.L) {
        case 1: fast::fwd_tile<1>(j, tx, ty, S, aes); break;
        case 2: fast::fwd_tile<2>(j, tx, ty, S, aes); break;
        case 3: fast::fwd_tile<3>(j, tx, ty, S, aes); break;
        case 4: fast::fwd_tile<4>(j, tx, ty, S, aes); break;
        default: fast::fwd_tile<5>(j, tx, ty, S, aes); break;
        }
        __syncthreads();
    }
}

static_assert(fast::Geom<1>::kT == tile_side(1) && fast::Geom<2>::kT == tile_side(2) &&
                  fast::Geom<3>::kT == tile_side(3) && fast::Geom<4>::kT == tile_side(4) &&
                  fast::Geom<5>::kT == tile_side(5),
              "tile_side() must match the tile bodies");

size_t tile_smem_bytes(uint32_t L)
{
    const int words = L <= 3 ? fast::Geom<3>::kWords : (L == 4 ? fast::Geom<4>::kWords : fast::Geom<5>::kWords);
    return sizeof(AesSmem) + 4 * (size_t)words;
}

cudaError_t launch_tiles(const Work &w, uint32_t grid, size_t smem, cudaStream_t stream)
{
    cudaError_t e = cudaFuncSetAttribute(tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    tile_kernel<<<grid, kThreads, smem, stream>>>(w);
    return cudaGetLastError();
}

cudaError_t tile_occupancy(size_t smem, int *blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, tile_kernel, kThreads, smem);
}

} // namespace frag
