/*
 * frag.h -- C ABI of the B300 library for agnostic data fragmentation with a
 * reversible integer wavelet (Chapter 5 of "An Efficient Data Protection
 * Architecture Based on Fragmentation and Encryption", arXiv 1803.04880).
 *
 * The method (Sec. 5.2.1-5.2.3): any bytes are read as the pixels of a gray
 * image of a chosen width; a reversible integer LeGall 5/3 2-D wavelet
 * transform (lifting steps Eq. 5.1 / 5.2, rows before columns, dyadic levels
 * on the LL band, Sec. 5.1.1) splits them into a small private fragment, the
 * final-level LL band, protected with AES-128 (here in CTR mode), and a public
 * fragment made of the detail bands.  The transform maps integers to integers,
 * so recovery is exact.
 *
 * Conventions shared by every call:
 *   - Status codes: every function returns frag_status; FRAG_OK is 0.  On an
 *     error a thread-local message is available from frag_get_error().  No C++
 *     exception crosses this boundary.
 *   - Memory: the caller owns every data buffer.  Pointers named d_* are CUDA
 *     DEVICE pointers of the current device; pointers named h_* are HOST
 *     pointers.  The library owns plans, keys, batches and its own small
 *     device tables; the scratch of a call comes stream-ordered from a
 *     memory pool of the library's on each device, which keeps up to 8 GiB
 *     of freed scratch for the next calls (so they map no device pages).
 *   - Streams: work is enqueued on the caller's stream (frag_stream, a
 *     cudaStream_t; NULL is the legacy default stream) and the call returns
 *     without waiting, except the h_* entry points, which wait for their own
 *     copies.  Launch errors are returned; errors raised while the kernels run
 *     surface through frag_sync_status().
 *   - Matrix: for n input bytes and a plan (W, L), the image has W columns and
 *     H = ceil(n / W) rows rounded up to a multiple of 2^L; bytes past n are
 *     zeros that are never materialised.  Level l has H_l = H >> l rows and
 *     W_l = W >> l columns.
 *   - Level shift: bytes b are transformed as b - 128 (Sec. 5.2.3 treats
 *     0..255 as -128..127).
 *   - Private fragment: LL_L as int16 little-endian, row-major, H_L * W_L
 *     values (2 * H_L * W_L bytes), XORed with the AES-128-CTR keystream whose
 *     counter block for 16-byte block b is nonce (8 bytes, big-endian) || b
 *     (8 bytes, big-endian), b counted from 0 at the fragment's first byte.
 *   - Public fragment: the detail bands as int16 little-endian, coarsest level
 *     first, HL_L, LH_L, HH_L, HL_{L-1}, ..., HH_1, each band H_l x W_l
 *     row-major (2 * (H * W - H_L * W_L) bytes in all).  HL is the top-right
 *     quadrant (high horizontal frequency), LH bottom-left, HH bottom-right.
 *   - nbytes, (W, L) and the nonce are caller metadata: the fragments do not
 *     record them.  Use one nonce per buffer under one key.
 *   - Buffers may have any byte alignment.
 */
#ifndef FRAG_H
#define FRAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FRAG_ABI_VERSION 2

typedef enum {
    FRAG_OK = 0,
    FRAG_EINVAL = 1,       /* a bad argument: null pointer, bad size or plan */
    FRAG_EUNSUPPORTED = 2, /* a filter or shape the library does not implement */
    FRAG_ENOMEM = 3,       /* a host or device allocation of the library failed */
    FRAG_ECUDA = 4,        /* a CUDA runtime call failed (message has the text) */
    FRAG_ETIMEOUT = 5,     /* a bounded device-side wait ran out */
    FRAG_EDEVICE = 6       /* a kernel recorded an error in the device error word */
} frag_status;

/* The only filter the thesis uses (Sec. 5.1.1: "Le Gall 5/3", lifting form
 * Eq. 5.1 / 5.2, update step with a plus sign as in JPEG 2000). */
typedef enum { FRAG_FILTER_LEGALL53 = 0 } frag_filter;

typedef struct frag_plan_s *frag_plan;
typedef struct frag_key_s *frag_key;
typedef struct frag_batch_s *frag_batch;
typedef struct CUstream_st *frag_stream; /* same type as cudaStream_t */

/* Version of this ABI (FRAG_ABI_VERSION). */
int frag_abi_version(void);

/* Plan = matrix width W and number of levels L (Sec. 5.2.1: the chunk is a
 * matrix of configurable size; Sec. 5.1.1: two levels in the thesis, L here).
 * FRAG_EINVAL if out is NULL, levels == 0, levels > 8, width == 0 or width is
 * not a multiple of 2^levels; FRAG_EUNSUPPORTED for any other filter.  Every
 * call takes 1..8 levels except the allocation-free one (at most 5) and the
 * block mode (at most 3). */
frag_status frag_plan_create(frag_plan *out, uint32_t width, uint32_t levels, frag_filter filter);
frag_status frag_plan_destroy(frag_plan plan);

/* Sizes for nbytes of input: rows H, private and public fragment bytes.
 * Any of the output pointers may be NULL.  nbytes == 0 gives all zeros.
 * FRAG_EINVAL if H would not fit in 32 bits. */
frag_status frag_plan_sizes(frag_plan plan, uint64_t nbytes, uint32_t *height,
                            uint64_t *private_bytes, uint64_t *public_bytes);

/* Schedule of the streaming kernel that every other protect / recover call
 * runs (the autotuner in the Python package sets it; 0 keeps the library's
 * choice).  seg_rows: level-0 rows per work unit, a power of two in 16..256
 * (raised to 2^levels when smaller); ctas: CTAs of the persistent grid at
 * most (0 = every CTA that fits on the device).  A batch takes each
 * buffer's seg_rows from that buffer's plan and the grid cap from its first
 * item's plan.  Results do not depend on the schedule.  FRAG_EINVAL for a
 * NULL plan or a seg_rows outside that set; get: either pointer may be NULL. */
frag_status frag_plan_set_schedule(frag_plan plan, uint32_t seg_rows, uint32_t ctas);
frag_status frag_plan_get_schedule(frag_plan plan, uint32_t *seg_rows, uint32_t *ctas);

/* Kernels that run the levels of a plan's protect / recover calls (batches
 * take each buffer's from that buffer's plan).  FRAG_PATH_AUTO (the default):
 * levels 1..min(L, 3) of a buffer run in one fused pass down its rows that
 * keeps LL_1 .. LL_{F-1} on chip, whenever the width is a multiple of 8, the
 * input (protect) or output (recover) is 8-byte aligned, the level-1 bands
 * are 8-byte and the level-2 and level-3 bands 4-byte aligned, and, when the
 * fused levels are all of them (protect), the private fragment is 4-byte
 * aligned (8-byte with one level); levels 4..6 of such a buffer run in a
 * second fused pass over LL_3 under the same conditions one level down.  The
 * levels above, and buffers that do not meet those conditions, run in the
 * dependency-ordered level kernel.  The private fragment is enciphered by the
 * AES-CTR launch after the levels (protect) and deciphered by it before them
 * (recover), or, with three or more levels in the level kernel, by cipher
 * units inside that kernel's launch.
 * FRAG_PATH_LEVELS: every level in the dependency-ordered kernel.
 * FRAG_PATH_FUSED_CIPHER: as AUTO, but when the fused passes reach level L
 * the last of them also enciphers LL_L with AES-128-CTR before storing it
 * (protect), or deciphers it right after loading it (recover, private
 * fragment 4-byte aligned, 8-byte with one fused level in that pass), so the
 * private fragment makes no extra trip through memory (measured slower than
 * AUTO on this GPU: the cipher's table lookups then share the fused kernel's
 * issue slots and shared memory).  Results do not depend on the path.
 * FRAG_EINVAL for a NULL plan or an unknown path; get: FRAG_EINVAL if path is
 * NULL. */
typedef enum {
    FRAG_PATH_AUTO = 0,
    FRAG_PATH_LEVELS = 1,
    FRAG_PATH_FUSED_CIPHER = 2
} frag_path;
frag_status frag_plan_set_path(frag_plan plan, frag_path path);
frag_status frag_plan_get_path(frag_plan plan, frag_path *path);

/* Block mode (Sec. 5.2.1: every chunk is processed block by block, 8 x 8 in
 * the thesis).  block = 0 (the default): the whole matrix is transformed.
 * block = B: every B x B block of the matrix is transformed as an image of
 * its own -- L levels inside the block, the symmetric extension at the
 * block's own borders, so no block depends on another.  H becomes ceil(n /
 * W) rounded up to a multiple of B, and the fragments keep the whole-matrix
 * layout: band (l, k) is an H_l x W_l int16 image in which block (bi, bj)
 * fills rows [bi B / 2^l, (bi + 1) B / 2^l) and columns [bj B / 2^l,
 * (bj + 1) B / 2^l); the private fragment is LL_L - 128 laid out the same way
 * and enciphered as always.  A chunk D_i of C x C bytes is a plan of width
 * C.  FRAG_EINVAL for a NULL plan, a width that is not a multiple of B or a
 * B below 2^L; FRAG_EUNSUPPORTED for B other than 0 or 8 (the CUDA path
 * implements the thesis's 8 x 8 blocks, up to 3 levels).  The
 * allocation-free call does not take block plans (FRAG_EUNSUPPORTED). */
frag_status frag_plan_set_block(frag_plan plan, uint32_t block);
frag_status frag_plan_get_block(frag_plan plan, uint32_t *block);

/* The thesis's storage of its three fragments (Sec. 5.2.1: the private, the
 * first and the second public and protected fragment; Sec. 5.2.3: 10 or 11
 * bits a coefficient), for 8 x 8 blocks at two levels only: packed != 0
 * makes frag_protect / frag_recover of this plan read and write
 *   private  A: per block LL_2 - 128 as 4 x 10 bits (5 bytes), blocks
 *              row-major, enciphered with the same AES-128-CTR;
 *   public   B then C: B holds per block HL_2 and LH_2 at 10 bits and HH_2
 *              at 11 (124 bits), the blocks of a block row every 124 bits,
 *              each block row starting on a byte; C per block HL_1, LH_1,
 *              HH_1 at 10 bits (60 bytes), blocks row-major.
 * A value is its two's complement in its width; a record's values follow
 * each other from bit 0 (each band's tile row-major, bands in the order
 * above) and fill bytes from the least significant bit.  The coefficient
 * bounds (Sec. 5.2.3) make the widths enough; a value outside its width
 * makes frag_sync_status report FRAG_EDEVICE.  frag_plan_sizes gives
 * |A| and |B| + |C|; frag_plan_fragment_sizes splits the public part.
 * Batched calls take packed plans beside any others.  FRAG_EUNSUPPORTED
 * unless the plan has levels == 2 and block 8; frag_plan_set_block on a
 * packed plan to anything but 8 is FRAG_EINVAL. */
frag_status frag_plan_set_packed(frag_plan plan, uint32_t packed);
frag_status frag_plan_get_packed(frag_plan plan, uint32_t *packed);

/* The three fragments of nbytes bytes under the plan (Sec. 5.2.1): sizes[0]
 * the private fragment, sizes[1] the first public and protected fragment
 * (the detail bands of level L, which lead the public fragment; B when
 * packed), sizes[2] the second (the other levels' bands; C when packed).
 * sizes[1] + sizes[2] is frag_plan_sizes' public_bytes.  FRAG_EINVAL if
 * sizes is NULL. */
frag_status frag_plan_fragment_sizes(frag_plan plan, uint64_t nbytes, uint64_t sizes[3]);

/* Keyed protection of the public fragments (Sec. 5.2.1: the private fragment
 * of a block and the key give, through SHA-256, the bit sequence XORed into
 * the first public and protected fragment; that protected fragment and the
 * key give, through SHA-512, the one XORed into the second).  On a packed
 * plan, on != 0 makes protect write, per 8 x 8 block idx = bi * (W / 8) + bj,
 *   B' = B XOR the first 124 bits of SHA-256(K || N || I || A record)
 *   C' = C XOR the first 480 bits of SHA-512(K || N || I || B' record)
 * with K the 16 AES key bytes, N the call's nonce and I = idx as 8 bytes
 * big-endian, the A record its 5 plaintext bytes and the B' record its 124
 * bits in 16 bytes (4 zero bits at the top); digest bit i (bit i % 8 of byte
 * i / 8) masks record bit i.  Recover takes SHA-512 of the stored B' first,
 * then SHA-256 of the deciphered A.  Sizes and the private fragment are
 * those of the packed plan.  The hashes run in the block kernel, on the
 * records in registers.  FRAG_EUNSUPPORTED unless the plan is packed;
 * frag_plan_set_packed(plan, 0) on a keyed plan is FRAG_EINVAL; FRAG_EINVAL
 * if on is NULL (get). */
frag_status frag_plan_set_protect_public(frag_plan plan, uint32_t on);
frag_status frag_plan_get_protect_public(frag_plan plan, uint32_t *on);

/* AES-128 key (Sec. 5.2.1 protects the private fragment with AES-128): the
 * round keys are expanded on the host (FIPS-197 Sec. 5.2) and kept resident on
 * each device that uses the key.  The 16 bytes are copied. */
frag_status frag_key_create(frag_key *out, const uint8_t key[16]);
frag_status frag_key_destroy(frag_key key);

/* Protect one buffer (Sec. 5.2.1, Fig. "SE process for the single block"):
 * d_in holds nbytes bytes; d_private receives private_bytes, d_public
 * public_bytes (see frag_plan_sizes).  Output buffers must not overlap the
 * input or each other.  nbytes == 0 is a no-op.  Asynchronous on stream. */
frag_status frag_protect(frag_plan plan, frag_key key, uint64_t nonce, const void *d_in,
                         uint64_t nbytes, void *d_private, void *d_public, frag_stream stream);

/* Recover one buffer (Sec. 5.2.3: the transform is lossless): the exact
 * inverse of frag_protect with the same plan, key, nonce and nbytes.  Writes
 * exactly nbytes bytes to d_out.  Fragments that were not produced with these
 * parameters give other bytes, never an out-of-bounds access. */
frag_status frag_recover(frag_plan plan, frag_key key, uint64_t nonce, const void *d_private,
                         const void *d_public, uint64_t nbytes, void *d_out, frag_stream stream);

/* Full-buffer AES-128-CTR: the thesis's full-encryption comparator for its
 * selective method (Sec. 5.4 and Chapter 4: the whole data encrypted with
 * AES-128, against which the fragmentation's speed is judged).  d_out[i] =
 * d_in[i] XOR keystream byte i, the keystream being AES-128 of the counter
 * blocks nonce (8 bytes big-endian) || block index (8 bytes big-endian) from
 * 0 -- the private fragment's cipher, so applying it twice gives the input
 * back.  Device buffers of nbytes bytes at any alignment (16-byte aligned
 * ones take 16-byte accesses); d_out may equal d_in (in place) but must not
 * overlap it otherwise.  nbytes == 0 is a no-op; FRAG_EINVAL if key is NULL
 * or a buffer is NULL with nbytes > 0.  Asynchronous on stream. */
frag_status frag_aes128_ctr(frag_key key, uint64_t nonce, const void *d_in, void *d_out,
                            uint64_t nbytes, frag_stream stream);

/* The same full-buffer AES-128-CTR computed bitsliced instead of with
 * tables (FIPS-197's rounds as AND/XOR circuits over bit planes of 32 blocks
 * a thread; the S-box as Boyar and Peralta's 128-gate circuit): the
 * measured alternative to the table form, which the library's fragment
 * cipher uses.  Same arguments, result, alignment and error behaviour as
 * frag_aes128_ctr; its output is byte-identical. */
frag_status frag_aes128_ctr_bitsliced(frag_key key, uint64_t nonce, const void *d_in, void *d_out,
                                      uint64_t nbytes, frag_stream stream);

/* Host-buffer forms of the two calls: copy the host input into stream-ordered
 * device memory (the library's pool), run the same kernels, copy the results
 * back, and return once they are in host memory.  Pinned (cudaHostAlloc) host
 * buffers give full copy bandwidth.  A buffer of 16 MiB or more whose levels
 * all run in the fused passes (1..6 levels, FRAG_PATH_AUTO) moves in row
 * bands of about 32 MiB (8 to 64 of them) on two library streams beside the
 * caller's: band k + 1 is copied in while band k is transformed and band
 * k - 1 copied out, so the two copy directions and the kernels overlap
 * (with pinned buffers).  At 4..6 levels the bands cover levels 1..3; the
 * levels above and the private fragment move whole, after the bands
 * (protect) or before them (recover).  The bytes written do not depend on
 * the form. */
frag_status frag_protect_host(frag_plan plan, frag_key key, uint64_t nonce, const void *h_in,
                              uint64_t nbytes, void *h_private, void *h_public,
                              frag_stream stream);
frag_status frag_recover_host(frag_plan plan, frag_key key, uint64_t nonce, const void *h_private,
                              const void *h_public, uint64_t nbytes, void *h_out,
                              frag_stream stream);

/* Batched forms: many independent buffers, each with its own plan, nonce and
 * size, under one key, processed by ONE persistent kernel launch whose CTAs
 * pull tiles from a device work queue ordered from the most to the least
 * costly buffer.  Each item's output is byte-identical to what the
 * single-buffer call gives for it.  The descriptors are copied into
 * library-owned memory before the call returns, so the caller may reuse the
 * array; that memory is released lazily once the launch has completed.
 * count == 0 is a no-op.  Items must not share output memory. */
typedef struct {
    frag_plan plan;
    uint64_t nonce;
    uint64_t nbytes;
    const void *d_in;
    void *d_private;
    void *d_public;
} frag_item;

typedef struct {
    frag_plan plan;
    uint64_t nonce;
    uint64_t nbytes;
    const void *d_private;
    const void *d_public;
    void *d_out;
} frag_ritem;

frag_status frag_protect_batch(const frag_item *items, uint32_t count, frag_key key,
                               frag_stream stream);
frag_status frag_recover_batch(const frag_ritem *items, uint32_t count, frag_key key,
                               frag_stream stream);

/* Batch objects for CUDA-graph capture: *_create builds the work queue and
 * uploads it (synchronously) to the current device; frag_batch_run enqueues
 * per wave only kernel launches -- the fused-level kernel for the buffers it
 * takes, a memset of the completion counters and queue head and one launch of
 * the dependency-ordered kernel for the remaining levels, and the AES-CTR
 * kernel for private fragments enciphered outside it -- so a capture of
 * frag_batch_run replays with no host work.  Buffers named in the items must
 * stay valid while the batch exists. */
frag_status frag_batch_create_protect(frag_batch *out, const frag_item *items, uint32_t count);
frag_status frag_batch_create_recover(frag_batch *out, const frag_ritem *items, uint32_t count);
frag_status frag_batch_run(frag_batch batch, frag_key key, frag_stream stream);
frag_status frag_batch_destroy(frag_batch batch);

/* What one frag_batch_run issues: *launches = kernel launches (up to three
 * per wave of buffers whose scratch fits the library's budget),
 * *scratch_bytes = device memory the batch holds for level scratch and
 * descriptors.  Either pointer may be NULL.  FRAG_EINVAL if batch is NULL. */
frag_status frag_batch_info(frag_batch batch, uint32_t *launches, uint64_t *scratch_bytes);

/* Per-kernel timing of a batch (instrumentation; off by default).  While
 * enabled, frag_batch_run records a CUDA event pair on the caller's stream
 * around each kernel launch.  frag_batch_launch_times waits for the recorded
 * events and adds, per kernel kind, the milliseconds between each pair to
 * ms[kind] and the number of launches to launches[kind] (both arrays of
 * FRAG_KERNEL_KINDS entries, zeroed first; either may be NULL), then
 * forgets the recorded pairs.  The events cost a few microseconds of host
 * time per run; they are not captured into CUDA graphs usefully, so disable
 * timing before capturing.  FRAG_EINVAL if batch is NULL. */
typedef enum {
    FRAG_KERNEL_FUSED = 0,  /* levels 1..3 in one pass down the rows */
    FRAG_KERNEL_LEVELS = 1, /* the dependency-ordered level kernel */
    FRAG_KERNEL_CIPHER = 2, /* AES-128-CTR over private fragments */
    FRAG_KERNEL_BLOCKS = 3, /* block mode (frag_plan_set_block) */
    FRAG_KERNEL_FUSED_LOW = 4, /* levels 4..6 in one pass over the level-3 LL */
    FRAG_KERNEL_KINDS = 5
} frag_kernel_kind;
frag_status frag_batch_set_timing(frag_batch batch, int enable);
frag_status frag_batch_launch_times(frag_batch batch, double *ms, uint32_t *launches);

/* Batched protect that allocates nothing.  The thesis has no counterpart:
 * this is a deployment aid.  Some callers may not call cudaMalloc at all --
 * a plug-in whose host process owns every byte of device memory through its
 * own pool, or a latency-critical path that cannot accept the implicit
 * synchronisation of a driver allocation.  This call gives fragments
 * byte-identical to frag_protect_batch.  Items whose levels all fit the first
 * fused pass (1..3 levels under FRAG_PATH_AUTO's width and alignment
 * conditions, whatever the plan's path) go through the same two launches as
 * that call (the fused pass, then the CTR pass over their private
 * fragments); the others (4 or 5 levels, or buffers that pass does not take)
 * through the tile kernel that keeps every level of a tile in shared memory,
 * so that no item needs level scratch.  Up to 5 levels.  The call keeps its
 * descriptors, work queue, round keys, AES tables and error word in one
 * static device array of about 375 KiB that every GPU loading this library
 * holds until the process exits; it calls no cudaMalloc, cudaFree or other
 * allocating routine, and takes the raw 16-byte key instead of a frag_key.
 * The launches take the library's adaptive units and the full device
 * (frag_plan_set_schedule is not used).
 * Limits and rules:
 *   - at most FRAG_NOALLOC_MAX_ITEMS items per call; more is FRAG_EINVAL with
 *     a message saying so;
 *   - the first call on a device sets that device up synchronously (it looks
 *     up the array's device address and copies the AES tables into it);
 *   - every call shares the one array and the array keeps the last call's
 *     contents; the call clears what must start at zero (the queue head) on
 *     the stream.  Calls whose work overlaps on the GPU (other streams, or no
 *     ordering between them) race on the array and give wrong results: order
 *     them on one stream;
 *   - a kernel error of these calls (an inconsistent descriptor found on the
 *     device) goes to an error word inside the same array, not to the word
 *     frag_sync_status reads: read it with frag_noalloc_sync_status, which
 *     allocates nothing either.  The word keeps the first code until it is
 *     read, across calls;
 *   - the array's contents (the AES tables the set-up copied) do not survive
 *     a reset of the device (cudaDeviceReset): do not call this after one in
 *     the same process.
 * The caller still owns and passes every input and output buffer. */
#define FRAG_NOALLOC_MAX_ITEMS 1024
frag_status frag_protect_batch_noalloc(const frag_item *items, uint32_t count,
                                       const uint8_t key[16], frag_stream stream);

/* The status read that goes with frag_protect_batch_noalloc (no counterpart
 * in the thesis either): waits for `stream`, then reads and clears the error
 * word in the static array of the current device with a synchronous copy
 * into static host memory -- no allocation.  FRAG_OK when no call's kernel
 * reported anything (or no call has run on this device), FRAG_EDEVICE with a
 * message naming the code when one did, FRAG_ECUDA if the wait or the copy
 * failed. */
frag_status frag_noalloc_sync_status(frag_stream stream);

/* Serving: protect / recover requests with continuous batching (the thesis
 * has no counterpart; it is the deployment form of the batched calls).
 *
 * A server owns a scheduler thread and max_groups streams on the current
 * device.  Submitting records the position of the caller's `ready` stream
 * (work queued there before the call, that fills the input, comes first)
 * and queues the request; it allocates nothing and returns at once with a
 * request id.  The scheduler admits waiting requests in arrival order while
 * their device memory -- outputs plus the library's level scratch, about
 * (private + public) / 3 -- fits memory_budget (0: free memory at creation
 * less 4 GiB; a request alone is always admitted, so none starves) and a
 * stream is free; allocates their outputs from a memory pool of the
 * server's own that keeps freed memory mapped for the next requests;
 * and launches the group as one frag_protect_batch and one
 * frag_recover_batch (at most max_items requests a group).  Requests that
 * arrive while groups run are admitted as streams and memory free up, so
 * their work overlaps on the device.  A host function after each group's
 * launches marks its requests done.  Every result is byte-identical to a lone
 * call's.  The caller keeps every input alive until its request is done.
 *
 * create: FRAG_EINVAL for a NULL argument, max_groups outside 1..16 or
 * max_items 0.  stop: finishes every submitted request and ends the thread;
 * wait, release and check still work, submit then fails.  destroy: stops,
 * then frees the outputs not released and the server.  submit: FRAG_EINVAL for a NULL argument
 * or a stopping server; errors of the plan as frag_plan_sizes gives them.
 * wait: blocks until the request is done (timeout_s < 0: no limit; else
 * FRAG_ETIMEOUT when it runs out), fills info (may be NULL) and returns the
 * status of the request's launch.  release: gives the request's outputs
 * back to the pool, ordered after the work on `after`; FRAG_EINVAL for an
 * unknown or unfinished request.  hold: while held (nonzero, counted), the
 * scheduler admits nothing; requests submitted meanwhile are admitted
 * together afterwards.  check: waits for the server's streams and reports
 * the device error word as frag_sync_status does. */
typedef struct frag_server_s *frag_server;
typedef struct {
    uint32_t done;            /* 1: the request's work has completed on the device */
    int32_t status;           /* FRAG_OK, or the error of its group's launch */
    void *d_private;          /* protect: the fragments the server allocated */
    void *d_public;
    uint64_t private_bytes, public_bytes;
    void *d_out;              /* recover: the recovered bytes the server allocated */
    uint64_t nbytes;          /* the request's buffer size */
    double t_submit, t_launch, t_done; /* seconds, the server's steady clock */
} frag_request_info;
frag_status frag_server_create(frag_server *out, frag_key key, uint64_t memory_budget, uint32_t max_groups,
                               uint32_t max_items);
frag_status frag_server_stop(frag_server server);
frag_status frag_server_destroy(frag_server server);
frag_status frag_server_submit_protect(frag_server server, frag_plan plan, uint64_t nonce, const void *d_in,
                                       uint64_t nbytes, frag_stream ready, uint64_t *id);
frag_status frag_server_submit_recover(frag_server server, frag_plan plan, uint64_t nonce,
                                       const void *d_private, const void *d_public, uint64_t nbytes,
                                       frag_stream ready, uint64_t *id);
frag_status frag_server_wait(frag_server server, uint64_t id, double timeout_s, frag_request_info *info);
frag_status frag_server_release(frag_server server, uint64_t id, frag_stream after);
frag_status frag_server_hold(frag_server server, int hold);
frag_status frag_server_stats(frag_server server, uint64_t *launches, uint64_t *used_bytes, uint32_t *pending,
                              uint32_t *in_flight);
frag_status frag_server_check(frag_server server);

/* Thread-local text of the last error (always NUL-terminated).  Returns
 * FRAG_OK, or FRAG_EINVAL if buf is NULL or len is 0. */
frag_status frag_get_error(char *buf, size_t len);

/* Waits for stream, then reads and clears the device error word of the
 * current device: FRAG_OK, FRAG_EDEVICE (a kernel found an inconsistent
 * descriptor), FRAG_ETIMEOUT (a bounded wait ran out) or FRAG_ECUDA. */
frag_status frag_sync_status(frag_stream stream);

/* Failure-path self-test (the thesis has no counterpart).  Every wait in the
 * library's kernels is bounded: a unit that waits for another unit's output,
 * or for a shared-memory stage, gives up after a fixed number of polls, sets
 * the device error word and returns, so a launch always ends and the context
 * stays usable.  This call enqueues on `stream` one such wait on a counter
 * that nothing increments, bounded at `polls` polls (each poll sleeps at most
 * about 1 us); the next frag_sync_status on the stream then returns
 * FRAG_ETIMEOUT.  FRAG_EINVAL if polls is 0. */
frag_status frag_check_wait_timeout(uint32_t polls, frag_stream stream);

/* The same for the wait of the fused kernel's TMA box loads: enqueues on
 * `stream` one wait, with that wait's code, on a shared-memory stage barrier
 * armed for 16 bytes that no copy delivers, bounded at `polls` polls of the
 * barrier; the next frag_sync_status on the stream then returns
 * FRAG_ETIMEOUT ("a bounded wait for a TMA box load ran out").  FRAG_EINVAL
 * if polls is 0. */
frag_status frag_check_box_wait_timeout(uint32_t polls, frag_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* FRAG_H */
