/*
 * fqbfs.h -- C ABI of the compressed-frontier BFS library (libfqbfs.so, CUDA, sm_103a).
 *
 * The library runs the data-parallel hot path of "Optimizing Communication by Compression for
 * Multi-GPU Scalable Breadth-First Searches" (arXiv 1704.00513) on one GPU: a level-synchronous,
 * direction-optimising BFS over a CSR graph in which every level's frontier is compressed with
 * delta coding + binary packing in blocks of 128 (the thesis' S4-BP128 choice, sec. 5.3),
 * measured in bytes, decompressed and consumed on the device -- the codec stage that the thesis
 * wraps around its two per-level exchanges (Algorithm 4: compress -> ALLGATHERV -> decompress,
 * compress -> ALLTOALLV -> decompress).
 *
 * Conventions for every call
 *  - Pointers named d_* are device pointers, h_* host pointers.  The caller owns every buffer.
 *    Streams are cudaStream_t values passed as void* (NULL = the legacy default stream).
 *  - Calls are asynchronous on the given stream unless stated otherwise.  Argument errors are
 *    returned before anything is enqueued.  Errors found by the device (unsorted input, a corrupt
 *    stream, a short output buffer) are written to the status record at the start of the
 *    workspace and read back with fq_work_status(), which synchronises the stream.
 *  - No call allocates device memory except fq_graph_create (which owns what it allocates until
 *    fq_graph_destroy).  Codec calls take a caller-provided workspace of fq_workspace_bytes().
 *  - Every device buffer passed to a codec call must be 16-byte aligned (the codec moves 128-bit
 *    vectors); a misaligned pointer returns FQ_EINVAL.
 *  - One workspace (or graph handle) must not be used by two calls that may overlap in time.
 *
 * Stream formats (all little-endian; sizes are multiples of 16 bytes)
 *  FQ, a strictly increasing uint32 sequence v[0..n) (a frontier queue, sec. 4.1.4):
 *    packed  {u32 'FQP1', n, nb = ceil(n/128), payload_words}, u32 base[nb], u8 b[nb],
 *            zeros to 16 B, then per block k the 128 slots at b_k bits each (4*b_k u32 words;
 *            slot j at bits [j*b_k, (j+1)*b_k), LSB first).  Slot 0 is 0 and base_k = v[128k]
 *            (frame of reference, Eq. 5); slot j >= 1 is v[128k+j] - v[128k+j-1] - 1 (delta
 *            coding, sec. 5.1); slots past n are 0; b_k = bit length of the block's largest
 *            slot (Eq. 6 read as a ceiling, Eq. 7).
 *    raw     {u32 'FQR1', n, 0, n}, u32 v[n], zeros to 16 B.
 *    The packed form is written only when strictly smaller than the raw one (sec. 5.1's
 *    losslessness requirement: the encoding must be smaller than the input; sec. 5.4.3 thresholds).
 *  FQX, the same sequence with patched exceptions (patched coding, sec. 5.1,
 *    Eq. 8-9; the PFOR family of sec. 5.3), written by fq_frontier_encode_px:
 *    {u32 'FQX1', n, nb, payload_words, E, 0, 0, 0}, u32 base[nb], u8 b[nb], u8 e[nb], zeros to
 *    16 B, the blocks' low b_k bits of every slot as in FQ, u8 slot[E] (each block's exception
 *    slots, increasing, 1..127), zeros to 16 B, u32 high[E] (slot value >> b_k), zeros to 16 B.
 *    Per block b_k minimises the block's bytes 16*b + 5*e_b, e_b = slots >= 2^b (ties to the
 *    larger b).  Written only when strictly smaller than the raw FQ form, which it writes
 *    otherwise.
 *  FB, a bitmap of N bits in uint64 words (bit i = bit i%64 of word i/64):
 *    {u32 'FBM1', u32 mode, u64 N} then either an FQ stream of the set positions (mode 1, when
 *    2*popcount <= N) or of the clear positions below N (mode 2), or -- when that is not
 *    strictly smaller -- the raw words with bits >= N cleared, zero-padded to 16 B (mode 0).
 */
#ifndef FQBFS_H
#define FQBFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
typedef int32_t fq_status;
#define FQ_OK 0
#define FQ_EINVAL 1     /* bad argument (NULL, misaligned, size out of range)             */
#define FQ_ENOMEM 2     /* fq_graph_create could not allocate its workspace                 */
#define FQ_ENOSPC 3     /* output capacity too small; the status detail is the size needed  */
#define FQ_ECORRUPT 4   /* a stream failed validation; the status detail locates the fault  */
#define FQ_EUNSORTED 5  /* encoder input not strictly increasing; detail = first bad index  */
#define FQ_ETIMEOUT 6   /* a bounded device-side wait gave up                               */
#define FQ_ECUDA 7      /* a CUDA runtime call failed                                       */
#define FQ_EBUSY 8      /* resource in use                                                  */

/* Human-readable name of a status code (static storage). */
const char *fq_status_string(fq_status s);

/* The last cudaError_t value a call of this library saw fail in the calling thread (0 if none);
 * *line (may be NULL) receives the library source line.  Explains an FQ_ECUDA return. */
int fq_last_cuda_error(int *line);

/* ------------------------------------------------------------------ sizes */

/* Largest FQ stream for n ids: 16 + pad16(4n) bytes (the raw form; packed is chosen only when
 * strictly smaller).  A capacity of this many bytes never yields FQ_ENOSPC. */
uint64_t fq_queue_bound(uint64_t n);

/* Largest FB stream for a bitmap of nbits bits: 16 + pad16(8 * ceil(nbits/64)) bytes. */
uint64_t fq_bitmap_bound(uint64_t nbits);

/* Workspace bytes for codec calls on up to max_ids ids and bitmaps of up to max_nbits bits.
 * The first 64 bytes hold the status record (struct fq_device_status). */
uint64_t fq_workspace_bytes(uint64_t max_ids, uint64_t max_nbits);

typedef struct fq_device_status {
    int32_t code;    /* fq_status of the last call that used this workspace              */
    uint32_t where;  /* internal stage that set it (0 = none)                            */
    uint64_t detail; /* ENOSPC: bytes needed; EUNSORTED: first bad index; ECORRUPT: a byte
                        or element index near the fault                                  */
} fq_device_status;

/* Synchronise `stream`, then read the status record of workspace d_work.  Returns its code
 * (FQ_OK if the device found nothing wrong); *h_detail (may be NULL) receives the detail.  The
 * record carries the outcome of the device-side checks that sec. 5.1's losslessness requirement
 * implies (a stream that does not decode to strictly increasing ids is rejected, never returned
 * silently wrong), and of Algorithm 5's compress/decompress steps run on the device, where no
 * host code sees the data. */
fq_status fq_work_status(const void *d_work, void *stream, uint64_t *h_detail);

/* ------------------------------------------------------------------ frontier queue codec */

/* Encode the strictly increasing ids d_ids[0..n) (n < 2^32) as an FQ stream at d_out
 * (capacity cap bytes).  The stream's size is written to the device u64 *d_out_bytes (0 on a
 * device-detected error; the needed size on FQ_ENOSPC).  Device errors: FQ_EUNSORTED,
 * FQ_ENOSPC.  The frontier queue compress step of Algorithm 4 (delta + binary packing, sec. 5.1, 5.3). */
fq_status fq_frontier_encode(const uint32_t *d_ids, uint64_t n, uint8_t *d_out, uint64_t cap,
                             uint64_t *d_out_bytes, void *d_work, uint64_t work_bytes, void *stream);

/* The same as fq_frontier_encode with the FQX (patched exceptions) format: a block whose largest
 * gaps are rare outliers keeps a small width and stores the outliers apart.  Same arguments,
 * workspace, bound (fq_queue_bound) and errors.  Patched coding, sec. 5.1. */
fq_status fq_frontier_encode_px(const uint32_t *d_ids, uint64_t n, uint8_t *d_out, uint64_t cap,
                                uint64_t *d_out_bytes, void *d_work, uint64_t work_bytes, void *stream);

/* Decode the FQ (or FQX) stream d_in[0..in_bytes) into d_ids (room for cap ids); the number of ids is
 * written to the device u64 *d_n.  The stream is validated (magic, nb, widths <= 32, sizes
 * against in_bytes, zero padding and slots, strictly increasing values without u32 overflow;
 * FQX also exception counts <= 127, none at width 32, exception slots increasing within the id
 * range, nonzero high parts that fit above the width);
 * a failure sets FQ_ECORRUPT.  Header-level faults are caught before any output is written;
 * value-level faults may leave d_ids partly written.  Never writes more than cap ids
 * (FQ_ENOSPC if the stream holds more).  Payloads reach shared memory by TMA bulk copies whose
 * waits are bounded: a copy that has not landed after the bound sets FQ_ETIMEOUT, and the warp
 * that waited lets its copies in flight land (bounded again) and stops, leaving d_ids partly
 * written.  The decompress step of the same algorithm. */
fq_status fq_frontier_decode(const uint8_t *d_in, uint64_t in_bytes, uint32_t *d_ids, uint64_t cap,
                             uint64_t *d_n, void *d_work, uint64_t work_bytes, void *stream);

/* ------------------------------------------------------------------ batched codec
 * S independent frontier segments in a fixed number of launches (4 to encode, 4 to decode,
 * whatever S is): the grouping of many small transfers into one that the thesis applies to its
 * exchanges (sec. 6.5, data-transfer grouping), applied to the codec.  Stream s is byte-for-byte
 * what fq_frontier_encode writes for segment s alone.
 *
 * Workspace: fq_batch_workspace_bytes(total_ids, S), 16-byte aligned; total_ids = seg_off[S]. */
uint64_t fq_batch_workspace_bytes(uint64_t total_ids, uint32_t S);

/* Segment s is d_ids[seg_off[s] .. seg_off[s+1]) (device u64 array of S+1 offsets, non-decreasing,
 * each segment strictly increasing and shorter than 2^32).  Stream s is written at
 * d_out + out_off[s] with capacity out_off[s+1] - out_off[s] (device u64 array of S+1 offsets,
 * each a multiple of 16; fq_queue_bound(length) per segment always suffices); its size lands in
 * d_out_bytes[s].  Device errors (status record of the workspace): FQ_EINVAL (bad segment table),
 * FQ_EUNSORTED (detail = global index of the first bad id), FQ_ENOSPC (detail = segment).  On an
 * error the contents of the affected streams are unspecified. */
fq_status fq_frontier_encode_batch(const uint32_t *d_ids, const uint64_t *d_seg_off, uint32_t S, uint64_t total_ids,
                                   uint8_t *d_out, const uint64_t *d_out_off, uint64_t *d_out_bytes, void *d_work,
                                   uint64_t work_bytes, void *stream);

/* Stream s is d_in[in_off[s] .. in_off[s] + in_bytes[s]) (in_off multiples of 16).  Its ids are
 * written to d_ids + seg_off[s], at most seg_off[s+1] - seg_off[s] of them; their count lands in
 * d_n[s].  Every stream is validated like fq_frontier_decode; a failure sets FQ_ECORRUPT (detail
 * = segment) and that segment's count to 0, the others are still decoded.  A tile payload copy
 * that outlasts its bounded wait sets FQ_ETIMEOUT (detail = tile), and that CTA stops decoding. */
fq_status fq_frontier_decode_batch(const uint8_t *d_in, const uint64_t *d_in_off, const uint64_t *d_in_bytes, uint32_t S,
                                   uint32_t *d_ids, const uint64_t *d_seg_off, uint64_t total_ids, uint64_t *d_n,
                                   void *d_work, uint64_t work_bytes, void *stream);

/* ------------------------------------------------------------------ encode without a workspace
 * The thesis has no counterpart to this entry point.  It serves callers that cannot allocate
 * device memory -- code running inside another framework's memory pool, which must not see
 * foreign cudaMalloc/cudaFree calls, or latency-critical paths that may not call the allocator
 * (it can synchronise the device).  It encodes exactly like fq_frontier_encode, but its scratch
 * is a fixed array inside the library's device image, reserved on every GPU that loads the
 * library until the process exits, so the caller passes only input, output and stream.
 *  - n must not exceed FQ_STATIC_MAX_IDS (2^24 ids); a larger n returns FQ_EINVAL and
 *    enqueues nothing.
 *  - The first call on a device looks up the array's device address once and caches it; make
 *    that first call before any stream capture on that device.
 *  - Every call uses the same array and it keeps the last call's contents: calls that may
 *    overlap on the GPU (other streams, other host threads) race and corrupt each other's
 *    output, so serialise them.
 *  - Device-detected errors show only in *d_out_bytes: 0 when the input is not strictly
 *    increasing; a value above cap (the size needed) when cap is too small.
 *  - Pointers must be 16-byte aligned.  No allocator is called. */
#define FQ_STATIC_MAX_IDS (1ull << 24)
fq_status fq_frontier_encode_static(const uint32_t *d_ids, uint64_t n, uint8_t *d_out, uint64_t cap,
                                    uint64_t *d_out_bytes, void *stream);

/* ------------------------------------------------------------------ bitmap codec */

/* Encode the bitmap d_words (ceil(nbits/64) words; bits >= nbits ignored) as an FB stream at
 * d_out (capacity cap); size to *d_out_bytes.  nbits <= 2^32.  Bitmap frontiers, sec. 3.1
 * (the popcount-indexed sparse vector), coded with the queue codec. */
fq_status fq_bitmap_encode(const uint64_t *d_words, uint64_t nbits, uint8_t *d_out, uint64_t cap,
                           uint64_t *d_out_bytes, void *d_work, uint64_t work_bytes, void *stream);

/* Decode the FB stream d_in[0..in_bytes) into d_words (ceil(nbits/64) words, every word
 * written; bits >= nbits cleared).  The header's N must equal nbits.  FQ_ECORRUPT on any
 * inconsistency, including a position >= N or raw tail bits set. */
fq_status fq_bitmap_decode(const uint8_t *d_in, uint64_t in_bytes, uint64_t *d_words, uint64_t nbits,
                           void *d_work, uint64_t work_bytes, void *stream);

/* ------------------------------------------------------------------ predecessor list
 * The BFS tree (depth, parent) as one container "FPL1", for the one exchange the thesis leaves
 * uncompressed: the predecessor reduction at the end of a BFS (sec. 4.1.4; its volume in the
 * results chapter exceeds that of all compressed frontier exchanges).  Layout (little-endian):
 *   u32 {"FPL1" = 0x314C5046, n, L, reached}; u64 off[2L]: stream k occupies [off[k], off[k+1])
 *   from the container's start, off[0] = 16 + 16 L, every stream a multiple of 16 bytes;
 *   streams 0 .. L-1: the level sets F_d = {v : depth[v] = d} in increasing order, each an FQ
 *   stream exactly as fq_frontier_encode writes it (F_0 = {root});
 *   streams L .. 2L-2: for d = 1 .. L-1, R_d[i] = the index of parent[F_d[i]] within F_{d-1},
 *   as an FR stream -- frame of reference without differencing (Eq. 5-6): packed
 *   {u32 "FRP1" = 0x31505246, n, nb = ceil(n/128), payload_words = 4 * sum(b)}, u32 min[nb],
 *   u8 b[nb] (b = bit length of the block's max - min), zero pad to 16, then per block 4*b words
 *   with slot j = value - min at bits [j*b, (j+1)*b) (slots past n zero); or raw
 *   {"FRR1" = 0x31525246, n, 0, n}, u32 values, zero pad to 16; packed only when smaller.
 * Sizes: fq_pred_bound(n, L) bytes always suffice; the workspace is fq_pred_workspace_bytes(n, L)
 * (about 21 bytes per vertex), 16-byte aligned, shared by encode and decode. */
uint64_t fq_pred_bound(uint64_t n, uint32_t levels);
uint64_t fq_pred_workspace_bytes(uint64_t n, uint32_t levels);

/* Encode the tree d_depth[n] (int32, -1 = unreached), d_parent[n] (uint32; parent[root] = root;
 * entries of unreached vertices are ignored) with `levels` = max depth + 1 into d_out (capacity
 * cap, 16-byte aligned); the container's size lands in the device u64 *d_out_bytes (0 on a device
 * error other than FQ_ENOSPC, the needed size on FQ_ENOSPC).  1 <= levels <= n < 2^32.  Device
 * errors (workspace status record): FQ_EINVAL with detail = vertex when a depth lies outside
 * [-1, levels), the depth-0 vertex is not its own parent, or a parent is not one level above its
 * child; FQ_EINVAL with detail = level when a level is empty or level 0 holds more than one vertex. */
fq_status fq_pred_encode(const int32_t *d_depth, const uint32_t *d_parent, uint64_t n, uint32_t levels, uint8_t *d_out,
                         uint64_t cap, uint64_t *d_out_bytes, void *d_work, uint64_t work_bytes, void *stream);

/* Decode the container d_in[0..in_bytes) (16-byte aligned) into d_depth[n] and d_parent[n]:
 * unreached vertices get depth -1 and parent 2^32 - 1.  The header's n must equal n; a container
 * of more than max_levels levels (the workspace's sizing) gives FQ_ENOSPC with detail = its L.
 * Validation (FQ_ECORRUPT): header, offset table, every stream's header and size, zero padding,
 * widths <= 32, matching level and rank counts, exactly one vertex at level 0, ids < n strictly
 * increasing within a level, no vertex at two levels, every rank below the size of the level above.
 * Faults in the header, the table or the streams leave d_depth and d_parent untouched; an id that
 * is out of order, out of range or repeated may leave them partly written. */
fq_status fq_pred_decode(const uint8_t *d_in, uint64_t in_bytes, int32_t *d_depth, uint32_t *d_parent, uint64_t n,
                         uint32_t max_levels, void *d_work, uint64_t work_bytes, void *stream);

/* ------------------------------------------------------------------ BFS */

typedef struct fq_graph fq_graph;

/* Wrap an undirected graph in CSR form: d_offsets[n+1] (int64, offsets[0] = 0,
 * offsets[n] = m), d_cols[m] (uint32 < n, each row sorted, symmetric, no self-loops) -- the
 * adjacency matrix A, held as compressed sparse rows, that Algorithm 2 multiplies with the
 * frontier (the synthetic graph of sec. 2.7.1, symmetrised as Graph 500 inputs are).  The handle
 * borrows both arrays (the caller keeps them alive and unchanged) and allocates its workspace
 * (about 30 bytes per vertex) on the current device: through the allocator installed with
 * fq_set_allocator when there is one, else cudaMalloc.  It also counts the vertices of degree 0
 * (reported as fq_bfs_stats.isolated).  n < 2^32.  Synchronous.
 * Errors: FQ_EINVAL (arguments), FQ_ENOMEM (the workspace or the pinned host record could not be
 * allocated; nothing is left allocated), FQ_ECUDA. */
fq_status fq_graph_create(const int64_t *d_offsets, const uint32_t *d_cols, uint64_t n, uint64_t m,
                          fq_graph **out);

/* Free a handle's workspace (synchronises the device first), through the allocator it was
 * allocated with. */
fq_status fq_graph_destroy(fq_graph *g);

/* Device memory for graph handles from the caller's own pool (the thesis has no counterpart:
 * this serves callers whose device memory must all come from one allocator, such as a framework's
 * caching pool).  alloc(bytes, ctx) returns a 256-byte aligned device pointer or NULL (the
 * create call then fails with FQ_ENOMEM and releases everything it took); release(ptr, bytes, ctx)
 * takes back what alloc gave.  Process-wide; applies to fq_graph_create calls made after it; each
 * handle remembers the allocator that allocated it.  NULL restores cudaMalloc/cudaFree. */
typedef struct fq_allocator {
    void *(*alloc)(uint64_t bytes, void *ctx);
    void (*release)(void *ptr, uint64_t bytes, void *ctx);
    void *ctx;
} fq_allocator;
fq_status fq_set_allocator(const fq_allocator *a);

#define FQ_TOP_DOWN 0
#define FQ_BOTTOM_UP 1

/* fq_bfs_opts.flags */
#define FQ_BFS_VISITED_STREAM 0x1u /* also encode the visited bitmap V_d every level          */
#define FQ_BFS_FORCE_TOP_DOWN 0x2u /* ignore the switching rule: top-down at every level        */
#define FQ_BFS_FORCE_BOTTOM_UP 0x4u/* bottom-up at every level after level 0                    */
#define FQ_BFS_TIMING 0x8u         /* time every kernel class with CUDA events (fills stats); each
                                      level's launches are then captured as a graph and launched
                                      whole, so the events see the kernels back to back rather than
                                      the host's submission of each one (host-driven loop only)  */
#define FQ_BFS_NO_CODEC 0x10u      /* skip the codec stage: expand the raw queue/bitmap (the plain
                                      BFS the codec stage is measured against; no streams)      */
#define FQ_BFS_PATCHED 0x40u       /* the per-level queue streams Q_d in the FQX format (patched
                                      exceptions, as fq_frontier_encode_px writes them) instead of FQ;
                                      B_d is then encoded from the bitmap rather than mirrored.  The
                                      top-down level decodes FQX like FQ.                          */
#define FQ_BFS_OVERLAP 0x80u       /* overlap the codec stage with the expansion (overlapped
                                      communication and software pipelining, sec. 6.5.2): each level
                                      expands the raw frontier (queue or bitmap) while, beside it on a
                                      second stream (host-driven loop) or a parallel graph branch
                                      (device-driven loop), Q_d and B_d are encoded and the form the
                                      direction consumes is decoded and compared with the raw one
                                      (FQ_ECORRUPT on any difference); the compaction waits for both.
                                      Depths, records, statistics and streams are those of the serial
                                      codec stage.  Ignored with FQ_BFS_NO_CODEC.                  */
#define FQ_BFS_DEVICE_LOOP 0x20u   /* run the level loop on the device: one CUDA graph (built on
                                      the first call per handle, output buffers and stream-log
                                      buffer, then reused) whose while node repeats the level and
                                      whose switch node picks the level body (encode form and
                                      direction, or the one-CTA codec stage of a small frontier),
                                      so no level waits on the host.  Same results, records and
                                      streams as the host-driven loop; FQ_BFS_TIMING is ignored
                                      (kernel_ms stay 0).  Needs a driver with conditional graph
                                      nodes (CUDA 12.4 or later).  The build captures streams:
                                      the library keeps handle creation and destruction in other
                                      threads from overlapping it; other code must not synchronise
                                      the whole device or free device memory meanwhile (build a
                                      handle's graph before starting concurrent work).           */

typedef struct fq_bfs_opts {
    uint32_t alpha; /* top-down -> bottom-up when m_f * alpha > m_u   (0 selects 14) */
    uint32_t beta;  /* bottom-up -> top-down when n_f * beta < n      (0 selects 24) */
    uint32_t flags;
    uint32_t min_codec_ids; /* compression threshold: a level whose frontier has fewer ids skips the
                               codec stage (its frontier is consumed raw; Q_d, B_d record 0 bytes and
                               are not logged); 0 codes every level.  Compression
                               thresholds, sec. 5.4.3 */
} fq_bfs_opts;

/* kernel classes reported by FQ_BFS_TIMING */
#define FQ_K_TOP_DOWN 0
#define FQ_K_BOTTOM_UP 1
#define FQ_K_COMPACT 2
#define FQ_K_ENCODE 3
#define FQ_K_DECODE 4
#define FQ_K_OTHER 5
#define FQ_NUM_KCLASS 6

typedef struct fq_bfs_stats {
    uint32_t levels;          /* non-empty levels = max depth + 1                               */
    uint32_t directions;      /* bit d set = level d expanded bottom-up (first 32 levels)       */
    uint64_t reached;         /* vertices with depth >= 0                                       */
    uint64_t reached_edges;   /* undirected edges inside the reached component (TEPS numerator) */
    uint64_t edges_examined;  /* adjacency entries read by the expansion kernels                */
    uint64_t raw_queue_bytes; /* sum over levels of 4 * n_f                                      */
    uint64_t enc_queue_bytes; /* sum over levels of |Q_d|                                        */
    uint64_t raw_bitmap_bytes;/* sum over levels of N/8 (frontier bitmaps)                       */
    uint64_t enc_bitmap_bytes;/* sum over levels of |B_d|                                        */
    uint64_t enc_visited_bytes;/* sum over levels of |V_d| (FQ_BFS_VISITED_STREAM)              */
    double kernel_ms[FQ_NUM_KCLASS];       /* FQ_BFS_TIMING: summed kernel time per class       */
    uint64_t kernel_launches[FQ_NUM_KCLASS];/* launches per class                               */
    uint64_t kernel_bytes[FQ_NUM_KCLASS];  /* algorithmic bytes per class (fq_bfs_level_bytes)  */
    uint64_t isolated;        /* vertices of degree 0 in the graph (never swept bottom-up)      */
} fq_bfs_stats;

typedef struct fq_level_record {
    uint32_t level;
    uint32_t direction;       /* FQ_TOP_DOWN or FQ_BOTTOM_UP used to expand this level          */
    uint64_t n_f;             /* |F_d|                                                          */
    uint64_t m_f;             /* sum of degrees over F_d                                        */
    uint64_t m_u;             /* sum of degrees over vertices not yet visited                   */
    uint64_t examined;        /* adjacency entries read while expanding F_d                     */
    uint64_t cols_read;       /* of those, the entries read from the column array: all of them
                                 top-down; bottom-up, those past the two that each vertex's
                                 16-byte head record holds (the handle keeps head records when
                                 the graph has fewer than 2^32 adjacency entries)               */
    uint64_t q_bytes, b_bytes, v_bytes; /* |Q_d|, |B_d|, |V_d| (0 when not encoded)             */
    uint64_t log_offset;      /* offset of Q_d, then B_d, then V_d in the stream log (or ~0)    */
    float kernel_ms[FQ_NUM_KCLASS]; /* FQ_BFS_TIMING, host-driven loop: this level's kernel time
                                       per class (0 otherwise)                                    */
} fq_level_record;

/* The design model of algorithmic bytes behind fq_bfs_stats.kernel_bytes, for one level: the bytes
 * each kernel class must move by its design (the numerator of its roofline fraction), from the level's
 * record, the graph's vertex and isolated-vertex counts, whether the root has degree 0,
 * `visited` = vertices visited once F_d is included (the sum of n_f over levels 0..d) and the
 * next frontier's size.  Writes out[FQ_NUM_KCLASS]; host only, needs no GPU.  Per class:
 *   encode    coded level: 4 n_f + |Q_d| + N/8 + |B_d|; V_d: N/8 + |V_d|;
 *   decode    top-down: |Q_d| + 4 n_f; bottom-up: |B_d| + N/8 (coded levels only);
 *   top_down  4 per edge examined + 20 per frontier vertex (offsets pair + queue id) + 8 per
 *             discovered vertex (depth, parent);
 *   bottom_up 4 N/8 (frontier, visited, isolated and next bitmaps) + 16 per unvisited vertex of
 *             nonzero degree (its offsets pair or head record; isolated vertices are skipped
 *             unread) + 4 per column entry read (cols_read) + 8 per discovered vertex;
 *   compact   3 N/8 + 20 per discovered vertex.
 * A coded level is one with q_bytes > 0; V_d is coded when v_bytes > 0. */
void fq_bfs_level_bytes(uint64_t n, uint64_t n_isolated, uint32_t root_isolated, const fq_level_record *rec,
                        uint64_t visited, uint64_t n_f_next, uint64_t *out);

/* Breadth-first search from root: the thesis' problem statement (sec. 4.1.2: input a source
 * vertex s, output the predecessor list) solved level-synchronously as in Algorithm 2 (the
 * frontier f multiplied by A, masked by the visited list, until f is empty), with the per-level
 * codec stage of Algorithm 4 / 5 (sec. 5.4.4: compress the frontier, measure, decompress) and the
 * direction optimisation of sec. 3.1.  Writes d_depth[n] (hop distance, -1 unreachable) and, if
 * d_parent is not NULL, d_parent[n] (a BFS tree: parent[root] = root, UINT32_MAX unreachable;
 * the validation rules of Algorithm 1 hold, sec. 2.6.3).
 * Level d: encode F_d as Q_d (queue) and B_d (bitmap) [and V_d], decide the direction from
 * (n_f, m_f, m_u), decode the form that direction consumes, expand it (top-down over the
 * decoded queue, or bottom-up against the decoded bitmap), compact the next frontier into a
 * sorted queue.  Stops when the next frontier is empty (the termination test of sec. 4.2.1).
 * Errors: FQ_EINVAL (arguments), FQ_ECORRUPT / FQ_ETIMEOUT (a per-level stream failed its
 * round trip, a bounded wait gave up), FQ_ENOSPC (stream log too small; the search itself is
 * complete), FQ_ECUDA.
 * h_stats (may be NULL) and h_levels[0..max_levels) (may be NULL) receive the per-run and
 * per-level records.  If d_stream_log is not NULL every level's Q_d, B_d [, V_d] are copied
 * there back to back (fails with FQ_ENOSPC when stream_log_cap is exceeded).
 * Synchronous.  The host-driven loop reads one counter record per level; with
 * FQ_BFS_DEVICE_LOOP the host only starts the graph and reads the records at the end.  At most
 * 4096 level records are kept in device-loop mode.  Not thread-safe per handle. */
fq_status fq_bfs_run(fq_graph *g, uint32_t root, int32_t *d_depth, uint32_t *d_parent, const fq_bfs_opts *opts,
                     fq_bfs_stats *h_stats, fq_level_record *h_levels, uint32_t max_levels, uint8_t *d_stream_log,
                     uint64_t stream_log_cap, void *stream);

/* ------------------------------------------------------------------ multi-source BFS
 * k <= 64 roots traversed together in one persistent cooperative kernel launch: each vertex holds
 * a 64-bit mask of the roots that reached it, and a level ORs the frontier masks of the
 * neighbours into the not-yet-seen bits (the thesis' SpMV frontier step, t = A (x) f masked by
 * the visited list, Algorithm 2, bit-sliced over the roots).
 * d_depth[i * n + v] (k x n, row-major int32) = hop distance of v from h_roots[i], -1 if
 * unreachable -- equal to fq_bfs_run's depth for that root.  The graph is the CSR of
 * fq_graph_create.  Scratch: fq_msbfs_scratch_bytes(n) bytes (about 36 bytes per vertex).
 * h_stats (may be NULL): levels, reached = sum over roots of reached vertices, reached_edges =
 * sum over roots of undirected edges inside each root's component, edges_examined.  Synchronous.
 * The level barriers wait with a bound; FQ_ETIMEOUT if one gives up.  The multi-source frontier
 * has no codec stage. */
uint64_t fq_msbfs_scratch_bytes(uint64_t n);

/* Test hook for the bounded waits of fq_bfs_run_multi (the thesis has no counterpart): while
 * extra_arrivals > 0, every level barrier waits for that many more CTAs than the grid holds, so
 * none releases and each wait gives up after spin_limit polls (0 keeps the built-in bound of
 * 2^24 polls, about 2 s); the call then returns FQ_ETIMEOUT with the GPU context intact.  It
 * exists so that tests can drive the timeout exit path without faulting anything.  Process-wide;
 * (0, 0) restores normal barriers.  FQ_EINVAL if extra_arrivals > 1024. */
fq_status fq_msbfs_barrier_test(uint32_t extra_arrivals, uint32_t spin_limit);
fq_status fq_bfs_run_multi(const int64_t *d_offsets, const uint32_t *d_cols, uint64_t n, const uint32_t *h_roots,
                           uint32_t k, int32_t *d_depth, void *d_scratch, uint64_t scratch_bytes,
                           fq_bfs_stats *h_stats, void *stream);

/* ------------------------------------------------------------------ serving
 * A continuous-batching server over resident graphs (the thesis has no serving layer; this is the
 * serving form of its BFS + codec hot path).  `slots` worker threads each own a CUDA stream, a
 * codec workspace and a BFS handle per resident graph.  Requests queue FIFO; the head request is
 * admitted when a slot is idle and its device footprint fits in the HBM budget next to the resident
 * graphs and the running requests.  An admitted request allocates its device buffers stream-ordered,
 * copies its host input in, runs, copies its result to the host buffers and frees -- so requests
 * that arrive while others are on the GPU start as slots and memory free up, and their copies and
 * kernels overlap.  Each request's result is the one the plain calls give alone. */
#define FQ_REQ_BFS 1     /* h_out: int32 depth[n] (out_cap >= 4n); h_out2 (optional): parent[n]   */
#define FQ_REQ_ENCODE 2  /* h_in: uint32 ids[in_count]; h_out: FQ stream (out_cap bytes)            */
#define FQ_REQ_DECODE 3  /* h_in: FQ stream of in_count bytes (multiple of 16); h_out: ids (out_cap) */

typedef struct fq_request {
    uint32_t kind;       /* FQ_REQ_*                                                             */
    uint32_t graph;      /* BFS: id from fq_server_add_graph                                     */
    uint32_t root;       /* BFS: source vertex                                                   */
    uint32_t flags;      /* BFS: fq_bfs_opts.flags                                               */
    const void *h_in;    /* host input (kept valid until done)                                   */
    uint64_t in_count;   /* ENCODE: ids; DECODE: bytes                                           */
    void *h_out;         /* host output                                                          */
    uint64_t out_cap;    /* bytes at h_out                                                       */
    void *h_out2;        /* BFS: parent output or NULL                                           */
    uint64_t out2_cap;
    uint64_t out_count;  /* result: BFS reached vertices; ENCODE stream bytes; DECODE ids        */
    uint64_t aux;        /* result: BFS undirected edges in the reached component                */
    fq_status status;    /* result                                                               */
    int32_t done;        /* set to 1 when the result is in place                                */
    double t_submit, t_start, t_end; /* fq_server_clock() seconds                                 */
} fq_request;

typedef struct fq_server fq_server;

/* max_codec_ids bounds the ids of one codec request (workspace size).  Starts the slot threads on
 * the current device. */
fq_status fq_server_create(uint64_t hbm_budget_bytes, uint32_t slots, uint64_t max_codec_ids, fq_server **out);
/* Finishes the queued requests, joins the workers, frees everything. */
fq_status fq_server_destroy(fq_server *s);
/* Make a CSR graph (device arrays, borrowed) resident; creates one BFS handle per slot. FQ_EBUSY
 * while requests run. */
fq_status fq_server_add_graph(fq_server *s, const int64_t *d_offsets, const uint32_t *d_cols, uint64_t n, uint64_t m,
                              uint32_t *graph_id);
/* Queue a request (the struct stays owned by the caller and valid until done).  FQ_ENOMEM if it can
 * never fit in the budget. */
fq_status fq_server_submit(fq_server *s, fq_request *r);
/* Wait up to timeout_s seconds for r; returns its status, or FQ_ETIMEOUT. */
fq_status fq_server_wait(fq_server *s, fq_request *r, double timeout_s);
fq_status fq_server_info(fq_server *s, uint64_t *resident, uint64_t *in_use, uint64_t *queued, uint64_t *completed);
/* The server's clock (seconds, monotonic) used for the request timestamps. */
double fq_server_clock(void);

/* ------------------------------------------------------------------ launch autotuning
 * Grid sizes of the launches whose best size depends on the GPU and the input size, settable per
 * size class (floor(log2(items)), 0..40) as CTAs per SM; 0 restores the built-in choice.  A tuner
 * (paper_1704_00513_gb300/autotune.py) times the candidates on synthetic inputs and caches the
 * winners in a JSON file.  The table is process-wide and read at each launch; a device-loop BFS graph
 * (FQ_BFS_DEVICE_LOOP) that baked the old grids is rebuilt on its next call. */
#define FQ_TUNE_ENC_WIDTHS 0u   /* encode, widths kernel (items: ids)                   */
#define FQ_TUNE_ENC_PACK 1u     /* encode, pack kernel (items: ids)                     */
#define FQ_TUNE_DEC_UNPACK 2u   /* decode, unpack kernel (items: ids)                   */
#define FQ_TUNE_BAT_ENCODE 3u   /* batched encode, widths and pack kernels (items: all ids) */
#define FQ_TUNE_BAT_DUNPACK 4u  /* batched decode, unpack kernel (items: all ids)       */
#define FQ_TUNE_BU_SWEEP 5u     /* BFS bottom-up sweep (items: vertices)                */
#define FQ_TUNE_TD_HUB 6u       /* BFS top-down hub items (items: vertices)             */
#define FQ_TUNE_NUM_SITES 7u
#define FQ_TUNE_MAX_CLASS 40u

/* FQ_EINVAL for an unknown site, a class above FQ_TUNE_MAX_CLASS or more than 32 CTAs per SM. */
fq_status fq_tune_set(uint32_t site, uint32_t size_class, uint32_t ctas_per_sm);
/* The value set for (site, class), 0 if none (or the arguments are out of range). */
uint32_t fq_tune_get(uint32_t site, uint32_t size_class);

#ifdef __cplusplus
}
#endif

#endif /* FQBFS_H */
