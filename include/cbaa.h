/*
 * cbaa.h -- C ABI of libcbaa.so, the sm_103a (B300) implementation of the
 * Cube of Bit Arrays Algorithm (CBAA) for super-host detection of Xu, Ding
 * and Hu, "GPU based Real-time Super Hosts Detection at Distributed Edge
 * Routers" (arXiv 1901.06207).
 *
 * Problem (Section III, Def. 1): in a time window, find every inner address
 * iip whose number of distinct outer peers |OP(iip)| is at least theta, from
 * <iip, oip> pairs seen at several edge routers, each router keeping a small
 * local structure that a global server merges.
 *
 * Conventions for every call:
 *  - Pointers named dev_* are CUDA device pointers (global memory of the
 *    current device); host_* are host pointers.  The caller owns all of
 *    them.  None of the calls below allocates device memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls marked "async" only enqueue work on it; calls marked
 *    "sync" return after the stream reached the end of their work.
 *  - Every call returns an int status (CBAA_OK = 0 or a negative error).
 *    On an error nothing is enqueued unless stated otherwise.
 *  - Calls are thread-safe as long as two calls never touch the same cube
 *    or workspace concurrently.
 *
 * Cube memory format (the bytes a local server sends, Section III.C): uint32
 * words.  With S = 2^r sketches, A = n_ra + n_va arrays, array a holding
 * c_a = 2^cbn[a] columns of g = 2^log2_g bits and W = g/32 words per column:
 *   word(cs, a, col, w) = cs*CSW + B_a + col*W + w,
 *   B_a = sum_{b<a} c_b*W,  CSW = sum_a c_a*W,
 * and row `row` of a column is bit (row % 32) of word (row / 32).
 */
#ifndef CBAA_H
#define CBAA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CBAA_MAX_ARRAYS 8   /* |RA| + |VA| */
#define CBAA_MAX_RA     6   /* |RA| */

/* Status codes. */
enum {
    CBAA_OK                 = 0,
    CBAA_ERR_INVALID_ARG    = -1,  /* bad geometry, null or misaligned pointer, short buffer */
    CBAA_ERR_GEOMETRY       = -2,  /* merge of cubes with different parameters (Section III.C) */
    CBAA_ERR_CAPACITY       = -3,  /* more hosts than the caller's output capacity */
    CBAA_ERR_WORKSPACE      = -4,  /* candidate tuples or hosts exceeded the workspace */
    CBAA_ERR_CUDA           = -5,  /* a CUDA runtime call failed */
    CBAA_ERR_TIMEOUT        = -6,  /* a bounded device wait gave up */
    CBAA_ERR_NO_DEVICE      = -7   /* no usable CUDA device */
};

/* Host-list flags. */
#define CBAA_FLAG_SATURATED 1u     /* union column had no zero bit; estimate uses Z = 1 */

/*
 * Geometry of a cube (Section III.A/B).
 *  r          CS selector width: the right (least significant) r bits of the
 *             mangled address select one of S = 2^r sketches; 1 <= r <= 16.
 *             The left part LP = mangled >> r has L = 32 - r bits.
 *  n_ra/n_va  number of restoring / validating arrays; 2 <= n_ra <= 6,
 *             n_ra + n_va <= 8.
 *  log2_g     rows per column g = 2^log2_g, 7 <= log2_g <= 15.
 *  cbn[a]     column-index width of array a (RA first, then VA); 5..16, and
 *             <= L for RAs.
 *  ring_off[i] (RA only) CL_bs(i) - r: CL(i) is cbn(i) consecutive bits of
 *             LP starting at this offset, wrapping from the top of LP to
 *             bit 0.  ring_off[0] = 0, strictly increasing, < L.  EP(i) runs
 *             from ring_off[i] to ring_off[i+1] (cyclically),
 *             |CP(i)| = cbn(i) - |EP(i)| >= 0 and |CP(i)| <= |EP(i+1)|
 *             (Section III.B).
 *  seed_*     seeds of the mangle (Section III.A), the row hash H_bv and the
 *             VA column hashes H_j (Alg. 1).  All three are the bijective
 *             32-bit finaliser x^=x>>16; x*=0x7feb352d; x^=x>>15;
 *             x*=0x846ca68b; x^=x>>16 applied to (input ^ seed); rows and
 *             VA columns take its top bits.
 *  threshold_form 0: hot-column bound g(1-eps)e^{-theta/g} (Thm. 2 solved
 *             for est >= theta); 1: the printed g(1+eps)e^{-theta/g} - g eps.
 */
typedef struct cbaa_params {
    uint32_t r, n_ra, n_va, log2_g;
    uint32_t cbn[CBAA_MAX_ARRAYS];
    uint32_t ring_off[CBAA_MAX_ARRAYS];
    uint32_t seed_mangle, seed_bv;
    uint32_t seed_va[CBAA_MAX_ARRAYS];
    uint32_t threshold_form;
} cbaa_params;

/* One detected super host (Alg. 3 output + Thm. 2 estimate). */
typedef struct cbaa_host {
    uint32_t ip;        /* restored, unmangled inner address */
    uint32_t z_union;   /* zero bits of its union column UC(ip) (Def. 2) */
    float    est;       /* -g ln(Z / (g - g eps)), Thm. 2 */
    uint32_t flags;     /* CBAA_FLAG_* */
} cbaa_host;

/* Outcome of a detect, written to device memory by cbaa_detect_async. */
typedef struct cbaa_detect_info {
    int32_t  status;        /* CBAA_OK, CBAA_ERR_CAPACITY or CBAA_ERR_WORKSPACE */
    uint32_t n_hosts;       /* hosts found (may exceed the output capacity) */
    uint32_t n_hot;         /* hot columns over all CS and RAs (Alg. 2) */
    uint32_t n_tuples;      /* partial tuples that passed the CP and union tests */
    uint32_t need_tuples;   /* on CBAA_ERR_WORKSPACE: entries needed by the stage that overflowed */
    uint32_t reserved[3];
} cbaa_detect_info;

/* Launch shapes of the update kernels (process-wide; see cbaa_set_tuning).
 * Zero fields take the defaults. */
typedef struct cbaa_tuning {
    uint32_t scatter_shape;        /* partitioned update, routing kernel: 0 = 512 threads x 8 packets,
                                      1 = 512 x 4, 2 = 1024 x 4, 3 = 256 x 8, 4 = 256 x 4,
                                      5 = 1024 x 8, 6 = 512 x 16, 7 = 256 x 16,
                                      8 = 1024 x 16 (row tiles; column tiles take 512 x 8) */
    uint32_t count_blocks_per_sm;  /* partitioned update, counting kernel grid (default 8) */
    uint32_t apply_items_per_sm;   /* partitioned update, tile-assembly items per SM (default 8) */
    uint32_t direct_blocks_per_sm; /* direct update grid (default 8 blocks of 256 threads) */
    uint32_t tile_kind;            /* partitioned update: 1 = column tiles (128 KiB runs of whole columns,
                                      one routed code per bit); row tiles (one row word of every column of
                                      a sketch, one routed record per packet; only where the geometry
                                      allows: sketch words / W <= 32768 and tiles <= 8192) with
                                      2 = run sizes from counting every packet, 3 = run capacities from
                                      counting every 16th tile of 1024 packets (records past a capacity
                                      are set by direct reductions; needs workspace room for an overflow
                                      list of every packet, else 2); 0 = 3 for passes of >= 8Mi packets,
                                      2 below, column tiles where row tiles are not allowed */
    uint32_t heavy;                /* partitioned update of one cube with row tiles: the heaviest sources'
                                      packets are set through one row bitmap per source in shared memory,
                                      the rest through row tiles.  0 = on for passes of >= 4Mi packets
                                      (128 KiB of bitmaps per block), 1 = off, 2 = on with 64 KiB of bitmaps
                                      (half as many sources), 3 = on with 128 KiB */
    uint32_t split_blocks;         /* heavy-source split: blocks of 1024 threads (at most one per SM),
                                      0 = one per SM (the shortest update).  Fewer leave SMs free for
                                      kernels on other streams, e.g. other windows' updates and detects in
                                      flight, at the cost of this update's time; at most 4096 */
} cbaa_tuning;

typedef struct cbaa_cube cbaa_cube;   /* opaque handle: a params copy plus the caller's memory */

/* Human-readable name of a status code.  Never returns NULL. */
const char *cbaa_status_str(int status);

/* Name of the last CUDA runtime error behind a CBAA_ERR_CUDA returned to
 * this host thread ("cudaSuccess" if none).  Never returns NULL. */
const char *cbaa_last_cuda_error(void);

/* Check a geometry against the rules above.  Host only, no device needed. */
int cbaa_params_validate(const cbaa_params *p);

/* Bytes of a cube with geometry p (0 if p is invalid).  Host only.
 * Section V.C's setting (r=4, 3+1 arrays, g = c = 2^12) gives 128 MiB. */
size_t cbaa_cube_bytes(const cbaa_params *p);

/* Bytes of detect workspace for up to max_candidates partial tuples and
 * hosts per stage (0 if p is invalid).  Host only. */
size_t cbaa_detect_workspace_bytes(const cbaa_params *p, size_t max_candidates);

/* Wrap caller memory as a cube and zero it (async).  dev_mem: >=
 * cbaa_cube_bytes(p) bytes, 16-byte aligned, owned by the caller for the
 * handle's lifetime.  *out receives a host-allocated handle. */
int cbaa_cube_init(const cbaa_params *p, void *dev_mem, size_t bytes, cbaa_cube **out, void *stream);

/* Free the handle (not the device memory).  NULL is accepted. */
int cbaa_cube_destroy(cbaa_cube *cube);

/* Device pointer of the cube words, and the geometry it was made with. */
void *cbaa_cube_data(const cbaa_cube *cube);
int cbaa_cube_params(const cbaa_cube *cube, cbaa_params *out);

/* Zero every bit (async): the start of a new time window. */
int cbaa_cube_reset(cbaa_cube *cube, void *stream);

/* The monitored (inner) network NI of Section III as CIDR prefixes.  An
 * edge router sees packets between NI and the outer network NO; the inner
 * address of a packet may be its source or its destination, since a super
 * host's peers are those it sends to or receives from (Def. 1). */
#define CBAA_MAX_INNER 16
typedef struct cbaa_inner_net {
    uint32_t n;                        /* prefixes in use, 0..CBAA_MAX_INNER */
    uint32_t addr[CBAA_MAX_INNER];     /* network address, host byte order */
    uint32_t len[CBAA_MAX_INNER];      /* prefix length 0..32 (0 matches every address) */
} cbaa_inner_net;

/* Attach NI to a cube (host only; takes effect for updates enqueued after
 * the call).  With n > 0 every update of this cube reads its pairs as raw
 * {src, dst}: a pair with exactly one address in NI becomes {that address,
 * the other} — its {iip, oip} — and a pair with both or neither address in
 * NI (not traffic between NI and NO) is skipped.  net = NULL or n = 0
 * restores the default, pairs given as {iip, oip}.  INVALID_ARG for n >
 * CBAA_MAX_INNER or a length above 32; the cube's bits are untouched.  A
 * multi-cube update requires the same NI on every cube. */
int cbaa_cube_set_inner_net(cbaa_cube *cube, const cbaa_inner_net *net);

/* Alg. 1 (Section III.B), async: for each of n pairs {iip, oip} at
 * dev_pairs (uint32[2n], 8-byte aligned; iip first) set bit H_bv(oip) in
 * the |RA|+|VA| columns that the mangled iip selects in its CS.  Bits are
 * only ever set, so any order of pairs and any concurrency give one cube.
 * n = 0 is a no-op. */
int cbaa_cube_update(cbaa_cube *cube, const uint32_t *dev_pairs, size_t n, void *stream);

/* Bytes of workspace that cbaa_cube_update_binned needs to route up to
 * max_pairs packets per pass (0 if p is invalid or its cube exceeds the
 * binned path's limit of 512 MiB).  Host only. */
size_t cbaa_update_workspace_bytes(const cbaa_params *p, size_t max_pairs);

/* Alg. 1 (Section III.B), async, partitioned: the same cube bits as
 * cbaa_cube_update, set without L2 atomics on hot columns.  Each bit set is
 * routed to the 128 KiB cube tile holding its word; tiles are assembled in
 * shared memory and ORed into the cube.  dev_ws: ws_bytes of caller device
 * memory (16-byte aligned), from cbaa_update_workspace_bytes; a workspace
 * sized for fewer than n packets is used in several passes.  Returns
 * CBAA_ERR_INVALID_ARG for cubes above 512 MiB or a workspace too small for
 * one packet. */
int cbaa_cube_update_binned(cbaa_cube *cube, const uint32_t *dev_pairs, size_t n, void *dev_ws, size_t ws_bytes,
                            void *stream);

/* The same as cbaa_cube_update_binned, except that the cube's words become
 * the bits of these n packets alone: its previous content is discarded, so
 * no cbaa_cube_reset is needed first (a window's first batch; the windows'
 * cube reused without a reset in between).  Where the heavy-source split
 * serves the pass (one cube, row tiles; see cbaa_tuning.heavy), the split's
 * blocks zero the cube while they read the packets (nothing writes the cube
 * before the split ends); on the other paths the cube is zeroed first by a
 * memset.  n = 0 zeroes the cube.  Errors as cbaa_cube_update_binned; on an
 * error nothing is enqueued. */
int cbaa_cube_update_binned_assign(cbaa_cube *cube, const uint32_t *dev_pairs, size_t n, void *dev_ws,
                                   size_t ws_bytes, void *stream);

/* Workspace for cbaa_cube_update_multi with n_cubes cubes of geometry p
 * and up to max_pairs packets per pass (0 if invalid, n_cubes > 16, or the
 * cubes together exceed 512 MiB).  Host only. */
size_t cbaa_update_multi_workspace_bytes(const cbaa_params *p, int n_cubes, size_t max_pairs);

/* Alg. 1 for several local cubes at once (the edge routers of Section
 * III.C), async: packets dev_pairs[j][0..n[j]) go to cubes[j].  One
 * partitioned pass covers all cubes, so uneven router loads share the whole
 * GPU.  All cubes must have the same geometry (else CBAA_ERR_GEOMETRY);
 * 1 <= n_cubes <= 16, together at most 512 MiB. */
int cbaa_cube_update_multi(cbaa_cube *const *cubes, int n_cubes, const uint32_t *const *dev_pairs, const size_t *n,
                           void *dev_ws, size_t ws_bytes, void *stream);

/* cbaa_cube_update_multi plus the global server's merge of Section III.C in
 * the same pass, async: every word the pass ORs into a router cube is ORed
 * into `global` too, so global |= the bits this pass sets in any router
 * cube (global = OR of the router cubes when they and global start empty),
 * with no separate merge pass reading the router cubes back.  global: same
 * geometry as the cubes (else CBAA_ERR_GEOMETRY), not one of them (else
 * CBAA_ERR_INVALID_ARG); same workspace as cbaa_cube_update_multi. */
int cbaa_cube_update_multi_merge(cbaa_cube *const *cubes, int n_cubes, const uint32_t *const *dev_pairs,
                                 const size_t *n, cbaa_cube *global, void *dev_ws, size_t ws_bytes, void *stream);

/* Set / read the process-wide launch shapes of the update kernels (for an
 * autotuner).  Results never depend on them.  Not synchronised with calls
 * running on other host threads: set them before launching work. */
int cbaa_set_tuning(const cbaa_tuning *t);
int cbaa_get_tuning(cbaa_tuning *t);

/* Section III.C merge, async: dst |= src_0 | ... | src_{k-1} word by word.
 * All cubes must share dst's geometry (else CBAA_ERR_GEOMETRY); k = 0 is a
 * no-op; dst may not be among srcs. */
int cbaa_cube_merge(cbaa_cube *dst, const cbaa_cube *const *srcs, int k, void *stream);

/* Section III.C merge into a fresh global cube, async: dst = src_0 | ... |
 * src_{k-1} word by word -- the merge with an all-zero initial value --
 * without reading dst, so no reset of dst is needed first (k = 0 zeroes
 * dst).  Same checks and errors as cbaa_cube_merge; all sources are checked
 * before anything is enqueued. */
int cbaa_cube_merge_assign(cbaa_cube *dst, const cbaa_cube *const *srcs, int k, void *stream);

/* Column statistics of the end-of-window pass, async (Eq. 1, Thm. 1 and the
 * hot-column bound of Section III.C):
 *   dev_zc   uint16[S][A][cmax]: zero bits of every column (cmax = max c_a;
 *            entries past c_a are left untouched),
 *   dev_za   uint64[S][A]: zero bits of every array,
 *   dev_eps  double[S]: eps = prod_a (ones_a / (c_a g)), the measured
 *            one-bit fraction standing in for Thm. 1's 1 - e^{-eta/(c g)},
 *   dev_zmax int64[S]: floor of the hot-column bound for theta.
 * Any of dev_zc, dev_eps, dev_zmax may be NULL; dev_za is required. */
int cbaa_column_stats(const cbaa_cube *cube, uint32_t theta, uint16_t *dev_zc, uint64_t *dev_za,
                      double *dev_eps, int64_t *dev_zmax, void *stream);

/* Alg. 2 + Alg. 3 + Thm. 2 (Section III.C), async: restore every address
 * whose union column has at most floor(theta_bn) zero bits, with its
 * estimate, sorted by ip.  dev_ws: cbaa_detect_workspace_bytes(p, m) bytes
 * (16-byte aligned) for some m; dev_out: room for cap records; dev_info:
 * one cbaa_detect_info.  The first min(n_hosts, cap) records (smallest ips)
 * are written.  Errors found on the device are reported in dev_info only. */
int cbaa_detect_async(const cbaa_cube *cube, uint32_t theta, void *dev_ws, size_t ws_bytes,
                      cbaa_host *dev_out, size_t cap, cbaa_detect_info *dev_info, void *stream);

/* Sharded restoration (Section III.C with the global server's work split
 * by sketch): cbaa_detect_async restricted to the sketches cs_lo <= cs <
 * cs_hi (cs = the right r bits of the mangled address).  Detection is
 * independent per sketch (each has its own eps and Zmax), so the host lists
 * of disjoint ranges covering [0, 2^r) together are exactly the full host
 * list.  INVALID_ARG unless cs_lo < cs_hi <= 2^r. */
int cbaa_detect_range_async(const cbaa_cube *cube, uint32_t cs_lo, uint32_t cs_hi, uint32_t theta, void *dev_ws,
                            size_t ws_bytes, cbaa_host *dev_out, size_t cap, cbaa_detect_info *dev_info,
                            void *stream);

/* The OR of Section III.C on raw words, async: dst[i] |= src_0[i] | ... |
 * src_{k-1}[i] for i < words.  For sharded merges, where each owner ORs
 * the slices of its sketches received from the other routers.  dst and
 * every src 16-byte aligned device pointers, words a multiple of 4, dst
 * not among srcs; k = 0 or words = 0 is a no-op. */
int cbaa_or_words(uint32_t *dst, const uint32_t *const *srcs, int k, size_t words, void *stream);

/* The global server's host list from its owners' (Section III.C split by
 * sketch), async: k host lists, each sorted by ip, in dev_blocks (block j =
 * dev_blocks[j * block_cap ...], its count in dev_infos[j].n_hosts, at most
 * block_cap used), merged into dev_out sorted by ip (the first out_cap
 * records).  The lists must hold disjoint addresses, as the owners of
 * disjoint sketch ranges do.  dev_info_out: the first status that is not
 * CBAA_OK (CBAA_ERR_CAPACITY also when the merged list exceeds out_cap), and
 * the sums of n_hosts, n_hot and n_tuples.  For all-gathered
 * cbaa_detect_range_async results, so that no host round trip is needed. */
int cbaa_merge_hosts(const cbaa_host *dev_blocks, size_t block_cap, int k, const cbaa_detect_info *dev_infos,
                     cbaa_host *dev_out, size_t out_cap, cbaa_detect_info *dev_info_out, void *stream);

/* Same as cbaa_detect_async followed by the copy of the records to host_out
 * (room for cap) and *n_out = number of hosts found; sync.  Returns
 * CBAA_ERR_CAPACITY when n_hosts > cap (the first cap records are valid) and
 * CBAA_ERR_WORKSPACE when the workspace was too small (*n_out then holds
 * the tuple count the overflowing stage needed). */
int cbaa_detect(const cbaa_cube *cube, uint32_t theta, void *dev_ws, size_t ws_bytes,
                cbaa_host *host_out, size_t cap, size_t *n_out, void *stream);

/* Largest detect scratch that cbaa_detect_static can use (bytes). */
#define CBAA_STATIC_SCRATCH_BYTES (16u << 20)

/* Detect without any device allocation, async.  The paper has no
 * counterpart: this exists for callers that cannot obtain device memory at
 * run time -- for example code running inside a host application that owns
 * all GPU memory through its own pool and forbids cudaMalloc, or a capture
 * agent with a fixed memory budget that must not grow while traffic flows
 * (cudaMalloc can also stall other work on the device or fail under memory
 * pressure from co-located processes).  It computes exactly what
 * cbaa_detect_async computes, but its scratch is a library-owned static
 * device array of CBAA_STATIC_SCRATCH_BYTES that every device loading the
 * library keeps until the process exits.  The caller still passes the
 * output records (dev_out, room for cap) and dev_info.
 *  - The first call on a device looks the array up on that device (make
 *    that device current, and make this first call before any stream
 *    capture).  The address found is kept for the life of the process, so
 *    do not use this entry point on a device after cudaDeviceReset (or
 *    any other teardown of its primary context): the kept address would
 *    no longer be valid there.
 *  - The call clears the scratch state it relies on, but all calls share
 *    one array: calls that overlap on the GPU (other streams, other host
 *    threads, the same device) race and give wrong results.
 *  - A geometry whose fixed tables do not fit returns CBAA_ERR_WORKSPACE
 *    before enqueuing anything; more candidate tuples than fit are reported
 *    in dev_info (status CBAA_ERR_WORKSPACE), as with cbaa_detect_async. */
int cbaa_detect_static(const cbaa_cube *cube, uint32_t theta, cbaa_host *dev_out, size_t cap,
                       cbaa_detect_info *dev_info, void *stream);

/* ---------------------------------------------------------------------
 * Learned estimator.  The paper estimates with Thm. 2 alone; these calls
 * add a small network that maps what the cube shows about an address to a
 * correction y of ln(1 + Thm. 2 estimate) towards ln(1 + |OP(ip)|), for
 * cubes whose arrays saturate.  Thm. 2 remains the fallback
 * (cbaa_learned_decide).
 *
 * Network: x (16 features) -> 64 ReLU -> 64 ReLU -> 1, weights in BF16,
 * activations and accumulation in FP32.  Parameters are one flat array in
 * the order W1[64][16], b1[64], W2[64][64], b2[64], W3[64], b3
 * (CBAA_MLP_PARAMS entries): BF16 (uint16 bit patterns) for the kernels,
 * FP32 for the optimiser's master copy.
 */
#define CBAA_MLP_IN     16
#define CBAA_MLP_HIDDEN 64
#define CBAA_MLP_PARAMS 5313

/* Features of n addresses (dev_ips), async, into dev_feats float[n][16]
 * (16-byte aligned): per array a < 4 the zero fraction of the address's
 * column (0..3), the zero fraction of the union column (4), the zero
 * fraction of array a of its sketch (5..8), eps (9), the Thm. 2 estimate / g
 * (10), ln(1 + estimate) / 10 (11), 1 if the union column is saturated
 * (12), the smallest column zero fraction (13), ln(ones fraction of the
 * union) minus the sum over all arrays of ln(ones fraction of the column)
 * (14; near 0 when the columns are unrelated, as for an address that never
 * appeared), ln(ones fraction of the union) (15); ones fractions are floored
 * at 1/g.  dev_za and
 * dev_eps come from cbaa_column_stats on the same cube. */
int cbaa_host_features(const cbaa_cube *cube, const uint64_t *dev_za, const double *dev_eps,
                       const uint32_t *dev_ips, size_t n, float *dev_feats, void *stream);

/* dev_y[s] = network(dev_x[s]) for s < n, async (dev_x float[n][16], 16-byte aligned). */
int cbaa_mlp_forward(const uint16_t *dev_w_bf16, const float *dev_x, size_t n, float *dev_y, void *stream);

/* Accumulate into dev_grad (float[CBAA_MLP_PARAMS]) the gradient, with
 * respect to the BF16 weights, of scale * sum_s (y_s - dev_t[s])^2, and add
 * sum_s (y_s - dev_t[s])^2 to *dev_loss; async.  The caller zeroes both. */
int cbaa_mlp_grad(const uint16_t *dev_w_bf16, const float *dev_x, const float *dev_t, size_t n, float scale,
                  float *dev_grad, float *dev_loss, void *stream);

/* One Adam step (Kingma and Ba) on the FP32 master weights with bias
 * correction for step >= 1, then the BF16 copy is refreshed; async. */
int cbaa_mlp_adam(float *dev_master, const float *dev_grad, float *dev_m, float *dev_v, uint16_t *dev_w_bf16,
                  float lr, float beta1, float beta2, float eps, uint32_t step, void *stream);

/* dev_w_bf16 = round-to-nearest-even BF16 of dev_master; async. */
int cbaa_mlp_to_bf16(const float *dev_master, uint16_t *dev_w_bf16, void *stream);

/* Training target per sample, async: dev_t[s] = ln(1 + dev_count[s]) -
 * ln(1 + est_s), the correction the network learns, with est_s the Thm. 2
 * estimate carried in the features (dev_feats float[n][16] from
 * cbaa_host_features) and dev_count the exact cardinality (the baseline of
 * Section V.A, 0 for an address never seen).  dev_count, dev_t float[n]. */
int cbaa_learned_target(const float *dev_feats, const float *dev_count, size_t n, float *dev_t, void *stream);

/* Super-host decision per address, async: card = exp(ln(1 + est) + y) - 1
 * with est the Thm. 2 estimate carried in the features, or est itself when
 * y is not finite; decision = card >= theta.  dev_card float[n],
 * dev_decision uint8[n]. */
int cbaa_learned_decide(const float *dev_y, const float *dev_feats, size_t n, uint32_t log2_g, float theta,
                        float *dev_card, uint8_t *dev_decision, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CBAA_H */
