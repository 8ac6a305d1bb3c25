// tile_kernels.cu -- fused multi-level LeGall 5/3 forward / inverse kernels
// with AES-128-CTR on the final LL band, for sm_103a.
//
// Each CTA is persistent: it loads the AES tables and round keys into shared
// memory once, then takes tiles (by a static stride, or from a device work
// queue in batched launches) until none are left.  A tile owns
// tile_w x tile_h level-0 pixels of one buffer; the CTA stages the tile plus
// its lifting halo in shared memory and runs every level in place there
// (Eq. 5.1 predict, Eq. 5.2 update, rows before columns within a level,
// Sec. 5.2.2), so each input byte is read from HBM once and each coefficient
// is written once.  In the in-place layout the level-l lattice is every
// 2^(l-1)-th sample: after level l the even / odd positions of that lattice
// hold the s (low) / d (high) values in each direction.
//
// The window is larger than the owned tile because the transform is global
// (symmetric extension only at the image border, Eq. 5.1's x_ext).  Values
// near the window edge are computed from incomplete neighbourhoods; they lie
// outside the dependency cone of the owned outputs and are never stored.
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

// Geometry of one tile window.  Lattice index i of level l-1 sits at level-0
// coordinate i << (l-1); the window origin is a multiple of 2^L (or 0), so
// every lattice starts on an even index.
struct Win {
    int64_t R0, R1, C0, C1; // owned rows / cols (level 0), half-open
    int64_t r0, r1, c0, c1; // window rows / cols (level 0), half-open
    int ld;                 // row pitch of the shared array (elements)
};

__device__ __forceinline__ int32_t &at(int32_t *S, const Win &w, int64_t row, int64_t col)
{
    return S[(row - w.r0) * w.ld + (col - w.c0)];
}

// One lifting step over the window along one axis, at lattice shift sh.
// Along the axis the lattice indices run lo..hi (lo even) and the signal
// length at this level is m; alo..ahi enumerate the lattice lines across.
enum Step { FWD_PREDICT, FWD_UPDATE, INV_UPDATE, INV_PREDICT };

template <Step STEP, bool HORIZONTAL>
__device__ void lift_step(int32_t *S, const Win &w, int sh, int64_t lo, int64_t hi, int64_t m,
                          int64_t alo, int64_t ahi)
{
    constexpr bool odd = (STEP == FWD_PREDICT || STEP == INV_PREDICT);
    const int64_t first = lo + (odd ? 1 : 0);
    if (hi < first)
        return;
    const int64_t per_line = (hi - first) / 2 + 1; // positions of this parity per line
    const int64_t total = per_line * (ahi - alo + 1);
    for (int64_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int64_t line = alo + idx / per_line;
        const int64_t i = first + 2 * (idx % per_line);
        auto P = [&](int64_t k) -> int32_t & {
            return HORIZONTAL ? at(S, w, line << sh, k << sh) : at(S, w, k << sh, line << sh);
        };
        if (odd) {
            // predict (Eq. 5.1) or its inverse; x[m] is the mirror x[m-2]
            int64_t ir = i + 1;
            if (ir > hi) {
                if (ir != m)
                    continue;
                ir = i - 1;
            }
            const int32_t t = (P(i - 1) + P(ir)) >> 1; // >> on int32 floors
            if (STEP == FWD_PREDICT)
                P(i) -= t;
            else
                P(i) += t;
        } else {
            // update (Eq. 5.2, plus sign) or its inverse; d[-1] is the mirror d[0]
            int64_t il = i - 1;
            if (i == 0)
                il = 1;
            else if (il < lo + 1)
                continue;
            const int64_t ir = i + 1;
            if (ir > hi)
                continue;
            // forward: the d at ir is final only if its right neighbour was there
            if (STEP == FWD_UPDATE && ir + 1 > hi && ir + 1 != m)
                continue;
            const int32_t t = (P(il) + P(ir) + 2) >> 2;
            if (STEP == FWD_UPDATE)
                P(i) += t;
            else
                P(i) -= t;
        }
    }
}

__device__ __forceinline__ bool make_window(const Job &j, uint32_t tx, uint32_t ty, bool fwd,
                                            Win &w)
{
    const int L = (int)j.L;
    const int64_t W = j.W, H = j.H;
    w.C0 = (int64_t)tx * j.tile_w;
    w.R0 = (int64_t)ty * j.tile_h;
    w.C1 = min(w.C0 + (int64_t)j.tile_w, W);
    w.R1 = min(w.R0 + (int64_t)j.tile_h, H);
    const int64_t hh = fwd ? (int64_t)halo_hi_fwd(L) : (int64_t)halo_hi_inv(L);
    w.c0 = max(w.C0 - (int64_t)halo_lo(L), (int64_t)0);
    w.r0 = max(w.R0 - (int64_t)halo_lo(L), (int64_t)0);
    w.c1 = min(w.C1 + hh, W);
    w.r1 = min(w.R1 + hh, H);
    w.ld = (int)(w.c1 - w.c0);
    return w.C0 < W && w.R0 < H;
}

// ---------------------------------------------------------------------------
// Forward tile: bytes -> details (public) + encrypted LL_L (private)
// ---------------------------------------------------------------------------
__device__ void fwd_tile(const Job &j, uint32_t tx, uint32_t ty, int32_t *S, const AesSmem &aes,
                         int *err)
{
    const int L = (int)j.L;
    const int64_t W = j.W, H = j.H;
    Win w;
    if (!make_window(j, tx, ty, true, w)) {
        if (threadIdx.x == 0)
            atomicCAS(err, 0, 1);
        return;
    }
    const int eh = (int)(w.r1 - w.r0);

    // map the bytes into the window; past n the byte is a virtual zero
    const int64_t cells = (int64_t)w.ld * eh;
    for (int64_t idx = threadIdx.x; idx < cells; idx += blockDim.x) {
        const int64_t r = idx / w.ld, c = idx - r * w.ld;
        const uint64_t g = (uint64_t)(w.r0 + r) * (uint64_t)W + (uint64_t)(w.c0 + c);
        S[idx] = g < j.n ? (int32_t)__ldg(j.in + g) : 0;
    }
    __syncthreads();

    for (int l = 1; l <= L; ++l) {
        const int sh = l - 1;
        const int64_t clo = w.c0 >> sh, chi = (w.c1 - 1) >> sh, mc = W >> sh;
        const int64_t rlo = w.r0 >> sh, rhi = (w.r1 - 1) >> sh, mr = H >> sh;
        // horizontal direction first (Sec. 5.2.2), then vertical
        lift_step<FWD_PREDICT, true>(S, w, sh, clo, chi, mc, rlo, rhi);
        __syncthreads();
        lift_step<FWD_UPDATE, true>(S, w, sh, clo, chi, mc, rlo, rhi);
        __syncthreads();
        lift_step<FWD_PREDICT, false>(S, w, sh, rlo, rhi, mr, clo, chi);
        __syncthreads();
        lift_step<FWD_UPDATE, false>(S, w, sh, rlo, rhi, mr, clo, chi);
        __syncthreads();

        // owned part of HL_l, LH_l, HH_l as int16 little-endian
        const int64_t y0 = w.R0 >> l, x0 = w.C0 >> l;
        const int64_t oh = (w.R1 - w.R0) >> l, ow = (w.C1 - w.C0) >> l, Wl = W >> l;
        const int64_t per_band = oh * ow;
        for (int64_t idx = threadIdx.x; idx < 3 * per_band; idx += blockDim.x) {
            const int b = (int)(idx / per_band);
            const int64_t rem = idx - b * per_band;
            const int64_t y = y0 + rem / ow, x = x0 + rem % ow;
            const int64_t lr = 2 * y + (b >= 1 ? 1 : 0), lc = 2 * x + (b != 1 ? 1 : 0);
            const int32_t v = at(S, w, lr << sh, lc << sh);
            uint8_t *dst = j.pub + band_offset(j.H, j.W, j.L, l, b) + 2 * (uint64_t)(y * Wl + x);
            dst[0] = (uint8_t)(v & 255);
            dst[1] = (uint8_t)((v >> 8) & 255);
        }
    }

    // private fragment: LL_L - 128 (the level shift moves only LL_L) as int16
    // little-endian, XORed with the AES-CTR keystream of its byte offsets
    const int64_t Y0 = w.R0 >> L, Y1 = w.R1 >> L, X0 = w.C0 >> L, X1 = w.C1 >> L;
    const int64_t WL = W >> L;
    const int64_t bpr = (2 * (X1 - X0) + 15) / 16 + 1;
    for (int64_t idx = threadIdx.x; idx < (Y1 - Y0) * bpr; idx += blockDim.x) {
        const int64_t y = Y0 + idx / bpr, jb = idx % bpr;
        const uint64_t start = 2 * (uint64_t)(y * WL + X0), end = 2 * (uint64_t)(y * WL + X1);
        const uint64_t blk = start / 16 + (uint64_t)jb;
        if (blk * 16 >= end)
            continue;
        uint32_t ks[4];
        aes_ctr_block(aes, j.nonce, blk, ks);
        for (int k = 0; k < 16; ++k) {
            const uint64_t o = blk * 16 + k;
            if (o < start || o >= end)
                continue;
            const int64_t x = (int64_t)(o / 2) - y * WL;
            const int32_t v = at(S, w, y << L, x << L) - 128;
            const uint32_t byte = (o & 1) ? ((uint32_t)v >> 8) & 255u : (uint32_t)v & 255u;
            j.priv[o] = (uint8_t)(byte ^ ks_byte(ks, k));
        }
    }
}

// ---------------------------------------------------------------------------
// Inverse tile: encrypted LL_L + details -> bytes
// ---------------------------------------------------------------------------
__device__ void inv_tile(const Job &j, uint32_t tx, uint32_t ty, int32_t *S, const AesSmem &aes,
                         int *err)
{
    const int L = (int)j.L;
    const int64_t W = j.W, H = j.H;
    Win w;
    if (!make_window(j, tx, ty, false, w)) {
        if (threadIdx.x == 0)
            atomicCAS(err, 0, 1);
        return;
    }

    // LL_L: decrypt the window's part of the private fragment, add back 128
    {
        const int64_t st = 1ll << L, WL = W >> L;
        const int64_t ylo = (w.r0 + st - 1) >> L, yhi = (w.r1 - 1) >> L;
        const int64_t xlo = (w.c0 + st - 1) >> L, xhi = (w.c1 - 1) >> L;
        const int64_t bpr = (2 * (xhi - xlo + 1) + 15) / 16 + 1;
        for (int64_t idx = threadIdx.x; idx < (yhi - ylo + 1) * bpr; idx += blockDim.x) {
            const int64_t y = ylo + idx / bpr, jb = idx % bpr;
            const uint64_t start = 2 * (uint64_t)(y * WL + xlo);
            const uint64_t end = 2 * (uint64_t)(y * WL + xhi + 1);
            const uint64_t blk = start / 16 + (uint64_t)jb;
            if (blk * 16 >= end)
                continue;
            uint32_t ks[4];
            aes_ctr_block(aes, j.nonce, blk, ks);
            for (int k = 0; k < 16; k += 2) {
                const uint64_t o = blk * 16 + k;
                if (o < start || o >= end)
                    continue;
                const uint32_t lo8 = __ldg(j.priv_in + o) ^ ks_byte(ks, k);
                const uint32_t hi8 = __ldg(j.priv_in + o + 1) ^ ks_byte(ks, k + 1);
                const int32_t v = (int32_t)(int16_t)(uint16_t)(lo8 | (hi8 << 8)) + 128;
                const int64_t x = (int64_t)(o / 2) - y * WL;
                at(S, w, y << L, x << L) = v;
            }
        }
    }
    // detail bands of every level at their lattice positions in the window
    for (int l = L; l >= 1; --l) {
        const int sh = l - 1;
        const int64_t Hl = H >> l, Wl = W >> l;
        const int64_t ylo = max((w.r0 >> l) - 1, (int64_t)0), yhi = min((w.r1 >> l) + 1, Hl - 1);
        const int64_t xlo = max((w.c0 >> l) - 1, (int64_t)0), xhi = min((w.c1 >> l) + 1, Wl - 1);
        const int64_t ny = yhi - ylo + 1, nx = xhi - xlo + 1;
        for (int64_t idx = threadIdx.x; idx < 3 * ny * nx; idx += blockDim.x) {
            const int b = (int)(idx / (ny * nx));
            const int64_t rem = idx - b * ny * nx;
            const int64_t y = ylo + rem / nx, x = xlo + rem % nx;
            const int64_t pr = (2 * y + (b >= 1 ? 1 : 0)) << sh;
            const int64_t pc = (2 * x + (b != 1 ? 1 : 0)) << sh;
            if (pr < w.r0 || pr >= w.r1 || pc < w.c0 || pc >= w.c1)
                continue;
            const uint8_t *src =
                j.pub_in + band_offset(j.H, j.W, j.L, l, b) + 2 * (uint64_t)(y * Wl + x);
            const uint32_t u = (uint32_t)__ldg(src) | ((uint32_t)__ldg(src + 1) << 8);
            at(S, w, pr, pc) = (int32_t)(int16_t)(uint16_t)u;
        }
    }
    __syncthreads();

    for (int l = L; l >= 1; --l) {
        const int sh = l - 1;
        const int64_t clo = w.c0 >> sh, chi = (w.c1 - 1) >> sh, mc = W >> sh;
        const int64_t rlo = w.r0 >> sh, rhi = (w.r1 - 1) >> sh, mr = H >> sh;
        // exact reverse of the forward level: columns first, then rows; within
        // a direction undo the update, then the predict
        lift_step<INV_UPDATE, false>(S, w, sh, rlo, rhi, mr, clo, chi);
        __syncthreads();
        lift_step<INV_PREDICT, false>(S, w, sh, rlo, rhi, mr, clo, chi);
        __syncthreads();
        lift_step<INV_UPDATE, true>(S, w, sh, clo, chi, mc, rlo, rhi);
        __syncthreads();
        lift_step<INV_PREDICT, true>(S, w, sh, clo, chi, mc, rlo, rhi);
        __syncthreads();
    }

    // owned bytes, only those before n
    const int64_t oh = w.R1 - w.R0, ow = w.C1 - w.C0;
    for (int64_t idx = threadIdx.x; idx < oh * ow; idx += blockDim.x) {
        const int64_t r = w.R0 + idx / ow, c = w.C0 + idx % ow;
        const uint64_t g = (uint64_t)r * (uint64_t)W + (uint64_t)c;
        if (g < j.n)
            j.out[g] = (uint8_t)at(S, w, r, c);
    }
}

// ---------------------------------------------------------------------------
// Persistent kernels
// ---------------------------------------------------------------------------
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
    if (w.jobs == nullptr) {
        local = t;
        return &w.single;
    }
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

template <bool FWD>
__global__ void __launch_bounds__(kThreads, 1) tile_kernel(Work w)
{
    extern __shared__ __align__(16) uint32_t smem[];
    AesSmem &aes = *reinterpret_cast<AesSmem *>(smem);
    int32_t *S = reinterpret_cast<int32_t *>(smem + sizeof(AesSmem) / 4);
    __shared__ unsigned long long s_tile;
    load_aes(aes, w);

    uint64_t t = blockIdx.x;
    for (;;) {
        if (w.queue != nullptr) {
            if (threadIdx.x == 0)
                s_tile = atomicAdd(w.queue, 1ull);
            __syncthreads();
            t = s_tile;
            __syncthreads();
        }
        if (t >= w.total_tiles)
            break;
        uint64_t local;
        const Job j = *find_job(w, t, local);
        if (j.tiles_x == 0 || local >= (uint64_t)j.tiles_x * j.tiles_y) {
            if (threadIdx.x == 0)
                atomicCAS(w.err, 0, 2);
            break;
        }
        const uint32_t tx = (uint32_t)(local % j.tiles_x), ty = (uint32_t)(local / j.tiles_x);
        if (j.path == 1) {
            fast::Smem &fs = *reinterpret_cast<fast::Smem *>(S);
            if (FWD) {
                if (j.L == 1)
                    fast::fwd_tile_fast<1>(j, tx, ty, fs, aes);
                else if (j.L == 2)
                    fast::fwd_tile_fast<2>(j, tx, ty, fs, aes);
                else
                    fast::fwd_tile_fast<3>(j, tx, ty, fs, aes);
            } else {
                if (j.L == 1)
                    fast::inv_tile_fast<1>(j, tx, ty, fs, aes);
                else if (j.L == 2)
                    fast::inv_tile_fast<2>(j, tx, ty, fs, aes);
                else
                    fast::inv_tile_fast<3>(j, tx, ty, fs, aes);
            }
        } else if (FWD) {
            fwd_tile(j, tx, ty, S, aes, w.err);
        } else {
            inv_tile(j, tx, ty, S, aes, w.err);
        }
        __syncthreads();
        if (w.queue == nullptr)
            t += gridDim.x;
    }
}

size_t tile_smem_bytes(uint32_t tile_w, uint32_t tile_h, uint32_t L, bool fwd)
{
    const uint32_t hh = fwd ? halo_hi_fwd(L) : halo_hi_inv(L);
    const size_t ew = tile_w + halo_lo(L) + hh, eh = tile_h + halo_lo(L) + hh;
    return sizeof(AesSmem) + ew * eh * sizeof(int32_t);
}

size_t fast_smem_bytes(bool fwd)
{
    (void)fwd;
    return sizeof(AesSmem) + sizeof(fast::Smem);
}

size_t job_smem_bytes(const Job &j, bool fwd)
{
    return j.path == 1 ? fast_smem_bytes(fwd) : tile_smem_bytes(j.tile_w, j.tile_h, j.L, fwd);
}

static const void *kernel_fn(bool fwd)
{
    return fwd ? (const void *)tile_kernel<true> : (const void *)tile_kernel<false>;
}

cudaError_t launch_tiles(bool fwd, const Work &w, uint32_t grid, size_t smem, cudaStream_t stream)
{
    cudaError_t e = cudaFuncSetAttribute(kernel_fn(fwd),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    if (fwd)
        tile_kernel<true><<<grid, kThreads, smem, stream>>>(w);
    else
        tile_kernel<false><<<grid, kThreads, smem, stream>>>(w);
    return cudaGetLastError();
}

cudaError_t tile_occupancy(bool fwd, size_t smem, int *blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(kernel_fn(fwd),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel_fn(fwd), kThreads,
                                                         smem);
}

} // namespace frag
