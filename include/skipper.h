/*
 * skipper.h -- C ABI of libskipper, Skipper maximal matching on one GB300.
 *
 * Skipper (Koohi Esfahani, "Skipper: Asynchronous Maximal Matching with a
 * Single Pass over Edges") resolves every edge of an undirected graph once,
 * by a just-in-time reservation on a per-vertex state that runs
 * ACC -> RSVD -> MCHD (Section IV-B, Fig. 4; Algorithm 1).  The result is a
 * maximal matching: no two output edges share an endpoint and every edge
 * touches an output edge (Section II-B).
 *
 * Graph input (Section II-A, the CSR definition N_v = neighbors[offsets[v] ..
 * offsets[v+1])): a CSR with n vertices and nnz stored entries,
 *   offsets  int64_t[n+1] in device memory, offsets[0] = 0, non-decreasing,
 *            offsets[n] = nnz;
 *   nbrs     uint32_t[nnz] in device memory, every id < n, base address
 *            16-byte aligned (the sweep reads it with 128-bit loads).
 * The library reads each stored entry (x, nbrs[i]) as the edge {x, nbrs[i]};
 * a graph stored once per direction (symmetric CSR) is the usual input, and
 * an edge stored for one endpoint only is matched all the same (Section V-C,
 * the paragraph on input formats and symmetrisation).  Self-loops are ignored (Algorithm 1
 * skips them).  Vertex ids are uint32 with n <= 0xFFFFFFFD.
 *
 * Output: mate uint32_t[n] in device memory, mate[v] = the vertex matched to
 * v, or MM_UNMATCHED.  Optionally the matched pairs (u, mate[u]) with
 * u < mate[u], in ascending u, as uint32_t[2*count].
 *
 * Ownership: the caller owns the CSR arrays and every output buffer; a
 * mm_graph handle only borrows the CSR, which must outlive it.  The handle
 * owns its scratch (state array, partition table, control words).
 *
 * Streams and errors: every call takes a CUDA stream (cudaStream_t passed as
 * void*, NULL = the legacy default stream) and is ordered on it.  Calls return
 * a status code and never throw; mm_last_error() gives a message for the last
 * failing call on the calling thread.  There is no CPU fallback: without a
 * CUDA device calls return MM_ERR_CUDA.
 */
#ifndef SKIPPER_H
#define SKIPPER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MM_UNMATCHED 0xFFFFFFFFu
#define MM_MAX_VERTICES 0xFFFFFFFDull

typedef enum mm_status {
    MM_OK = 0,
    MM_ERR_ARG = 1,          /* null pointer, bad size, bad alignment, bad option */
    MM_ERR_OOM = 2,          /* device memory for the handle's scratch could not be had */
    MM_ERR_CUDA = 3,         /* a CUDA call failed (includes: no device) */
    MM_ERR_TIMEOUT = 4,      /* a wait on a reserved vertex exceeded spin_limit polls */
    MM_ERR_BAD_GRAPH = 5,    /* CSR check failed, or a neighbour id >= n was met */
    MM_ERR_UNSUPPORTED = 6,  /* option combination not supported */
    MM_PENDING = 7           /* mm_server_wait: the request has not completed yet */
} mm_status;

/* mm_create_csr flags */
#define MM_CHECK_CSR 1u      /* check offsets and ids on the device (synchronous) */
#define MM_HOST_MAPPED 2u    /* the input arrays are page-locked host memory, read in place */
#define MM_BATCH_LOCAL_IDS 4u /* a packed batch whose member graphs keep local ids (see
                                 mm_skipper_batched); n may exceed MM_MAX_VERTICES */

typedef struct mm_graph mm_graph;

/*
 * Options of one matching call.  mm_default_options() fills the defaults;
 * zero in a field also selects its default.
 */
typedef struct mm_options {
    uint32_t status_bits;    /* 8: one state byte per vertex, 4 packed in a word
                                (the paper's one byte per vertex, Section IV-C);
                                2: the same three states in 2 bits, 16 vertices
                                a word (a quarter of the paper's footprint);
                                32: one word per vertex that is also the mate
                                entry (ACC = MM_UNMATCHED, RSVD = 0xFFFFFFFE,
                                matched = partner id).  0 = 8. */
    uint32_t serial;         /* 1: one GPU thread walks rows in ascending order and
                                neighbours in stored order (per graph in batched
                                mode); the result equals sequential greedy MM. */
    uint32_t grain;          /* merge-path items (rows + entries; edges for an edge
                                list) per work unit.  Must be a multiple of 128
                                when set.  0 = chosen from the graph: about two
                                units per resident sweep warp, the nearest power
                                of two in [512, 8192] (up to 32768 for
                                MM_HOST_MAPPED handles, whose units each start by
                                waiting on the host link).  mm_skipper_multi and
                                mm_skipper_static take 0 as 2048. */
    uint32_t block_threads;  /* sweep threads per block, multiple of 32, <= 512;
                                0 = 512 */
    uint32_t blocks_per_sm;  /* sweep blocks per SM; 0 = the occupancy maximum of the
                                instance used by default.  The plain and symmetric
                                CSR sweeps (single graph and batched) come in two
                                instances: compiled for 40 registers a thread (3
                                blocks of 512 threads, 48 warps per SM) and for 32
                                (4 blocks of 512, 64 warps per SM).  By default the
                                32-register one runs when the state array (the
                                packed states, or the mate array in the 32-bit
                                layout) takes at most half of the device's L2: it
                                then stays in L2, and more warps hide more
                                latency; a larger array's random sectors already
                                load the memory system, and more warps only queue
                                on it.  A value above what the 40-register instance
                                fits selects the 32-register one. */
    uint32_t nosync;         /* 1: return without waiting for the GPU; the status
                                of the work (timeout, bad id) is read by mm_sync() */
    uint32_t timing;         /* 1: record CUDA events around each kernel on the
                                call's stream (no extra wait); read back with
                                mm_get_timing() / mm_timing_history() */
    uint32_t use_graph;      /* mm_skipper_batched: 1 = launch through a CUDA graph
                                captured once per handle and option set */
    uint32_t l2_persist;     /* 1: L2 access-policy window (persisting) over the
                                state array for the sweep; 0 = per-load hints only */
    uint32_t stats;          /* 1: count reads, attempts and JIT conflicts in the
                                sweep (slower kernel instance); read back with
                                mm_get_stats() */
    uint64_t spin_limit;     /* polls of one wait before the call fails with
                                MM_ERR_TIMEOUT; 0 = 1 << 20 */
    uint64_t poison_vertex;  /* fault injection for tests: v + 1 leaves vertex v
                                RESERVED by no thread after initialisation, so
                                every wait on it runs out; 0 = off */
    uint32_t symmetric;      /* 1: the caller asserts that the CSR is symmetric (every
                                edge stored in the rows of both endpoints).  The
                                parallel sweep then tests each edge once, from the
                                row of its lower endpoint, and leaves entries (x, y)
                                with y < x to row y (Section V-C: one pass over the
                                edges needs each edge once); this halves the state
                                reads.  On a CSR that is not symmetric the result
                                is in general not maximal.  Serial mode and the
                                edge-list and multi-graph calls ignore it.  0 = off. */
    uint32_t id_loads;       /* when the parallel CSR sweep loads a chunk's neighbour
                                ids: MM_ID_LOADS_EAGER issues every 128-bit load of
                                the chunk before the row search (the load overlaps
                                it; quads whose rows are all known matched are
                                loaded and dropped); MM_ID_LOADS_SELECTIVE searches
                                first and loads only quads holding an entry of a
                                row not known matched (fewer bytes, the load after
                                the search).  MM_ID_LOADS_AUTO (0): selective for
                                MM_HOST_MAPPED handles, whose reads cross the host
                                link, eager otherwise.  The result is a maximal
                                matching either way.  Statistics instances
                                (stats = 1), batched calls and edge-list
                                handles load eagerly; mm_skipper_multi loads
                                eagerly unless asked for selective loads (the
                                server asks for them in every launch that reads
                                a request in place).  Other values give
                                MM_ERR_ARG. */
    uint32_t stage_windows;  /* 1: the parallel CSR sweep of mm_skipper stages each
                                32-row window (its row ends and state words) in
                                shared memory with a bulk copy (TMA) issued one
                                window ahead, instead of loading them when the
                                window starts.  Used for the 2- and 8-bit layouts
                                over a 16-byte aligned device CSR without
                                statistics or selective loads; ignored otherwise.
                                Off by default: on GB300 it is slower (the sweep
                                is bound by instruction issue, and the staged
                                state words are one window old).  0 = off. */
    uint32_t warps_per_graph; /* batched calls: at most this many work units per member
                                graph, so at most this many warps walk one graph at a
                                time (each graph's rows + entries are split evenly
                                over min(warps_per_graph, ceil(items / grain))
                                units); 0 = no cap (units of `grain` items). */
    uint32_t unit_order;     /* the order in which the parallel CSR sweeps (single
                                graph and batched) hand out their work units:
                                MM_ORDER_ASCENDING -- unit after unit from the
                                first row, so the units in flight form one band of
                                consecutive rows; MM_ORDER_DISPERSED -- the units
                                are cut into as many contiguous runs as the grid
                                has warps, and the k-th unit handed out is unit
                                k / runs of run k mod runs, so the units in flight
                                sit at evenly dispersed positions and each run is
                                walked in order (the GPU form of the paper's
                                threads that start at dispersed positions and
                                walk contiguous runs of blocks, Section IV-C).
                                Dispersed runs leave fewer rows unmatched when
                                their turn comes on graphs whose rows are mostly
                                open (uniform, grids) and cut the waits on ids
                                with locality; the single band keeps the memory
                                traffic of concurrent units close together.
                                MM_ORDER_AUTO (0): dispersed when the state array
                                takes at most half of the L2 (see blocks_per_sm),
                                ascending otherwise.  Other values: MM_ERR_ARG. */
    uint32_t reserved32;
    uint64_t reserved[1];
} mm_options;

#define MM_ORDER_AUTO 0u
#define MM_ORDER_ASCENDING 1u
#define MM_ORDER_DISPERSED 2u

#define MM_ID_LOADS_AUTO 0u
#define MM_ID_LOADS_EAGER 1u
#define MM_ID_LOADS_SELECTIVE 2u

/* Per-kernel device times of the last call made with options.timing = 1. */
typedef struct mm_timing {
    float init_ms;           /* state initialisation + merge-path partition */
    float sweep_ms;          /* the single pass over the entries (Algorithm 1) */
    float compact_ms;        /* pair-list compaction (0 when not requested) */
    float total_ms;          /* first event to last event */
    uint64_t units;          /* merge-path work units of the sweep */
    uint64_t reserved[3];
} mm_timing;

/*
 * Sweep statistics of the last mm_skipper call made with options.stats = 1.
 * A conflict is a failed CAS at Algorithm 1 line 11 or 14 (Section VI-E,
 * Table II); a CAS on a packed word that lost only to a neighbouring vertex's
 * field is retried and not counted.  hist[] counts entries by their number of
 * conflicts in Table II's bins: 1, 2, 3-4, 5-8, 9-16, 17-32, 33-64, 65-128,
 * 129-256, >256.
 */
typedef struct mm_stats {
    uint64_t entries_read;      /* neighbour ids the sweep loaded (matched rows are not read) */
    uint64_t windows;           /* 32-row windows loaded */
    uint64_t chunks;            /* chunks of up to 128 entries */
    uint64_t attempts;          /* entries that reached line 11 */
    uint64_t matches;           /* successful claims at line 14 */
    uint64_t conflicts;         /* failed CAS at lines 11 and 14 */
    uint64_t conflicted_entries;
    uint64_t max_conflicts;     /* on one entry */
    uint64_t hist[10];
    uint64_t transitions[4];    /* state transitions made (Fig. 4): ACC->RSVD (line 11),
                                   ACC->MCHD (line 14), RSVD->MCHD (line 15),
                                   RSVD->ACC (line 18); the holder's two are checked
                                   on the word their atomic returns */
    uint64_t illegal_transitions;  /* commits / releases that did not find RSVD (0) */
    uint64_t id_loads;          /* 128-bit neighbour-id loads (4 ids each) issued */
    uint64_t id_loads_open;     /* of those, the ones holding an entry of a row not
                                   known matched: the loads MM_ID_LOADS_SELECTIVE
                                   issues at the same point of the walk */
} mm_stats;

/*
 * Verdict of mm_validate (the exact checker, Section II-B).  flags == 0 means
 * mate is a maximal matching of the graph and the pair list (when given)
 * lists exactly its pairs.  Counting rules:
 *   for every v with m = mate[v] != MM_UNMATCHED:
 *     m >= n or m == v     -> n_bad_range, v is a bad vertex
 *     otherwise n_matched += 1, and
 *       mate[m] != v       -> n_asym,    v is a bad vertex
 *       m is not in row v and v is not in row m -> n_nonedge, v is a bad vertex
 *   n_pairs = #{v : m = mate[v] in range, v < m, mate[m] == v}
 *   each entry i of row x with y = nbrs[i] != x, mate[x] and mate[y] both
 *     MM_UNMATCHED -> n_uncovered (first_uncovered = smallest such i)
 *   pair list: (a, b) is valid when a < b < n, mate[a] == b, mate[b] == a;
 *     n_pairs_bad = invalid pairs + repeats of valid pairs; MM_V_PAIRS is set
 *     when n_pairs_bad > 0 or count != n_pairs.
 * first_bad_vertex / first_uncovered are UINT64_MAX when there is none.
 */
#define MM_V_RANGE     1u
#define MM_V_ASYM      2u
#define MM_V_NONEDGE   4u
#define MM_V_UNCOVERED 8u
#define MM_V_PAIRS     16u

typedef struct mm_verdict {
    uint32_t flags;
    uint32_t pad;
    uint64_t n_matched;
    uint64_t n_pairs;
    uint64_t n_bad_range;
    uint64_t n_asym;
    uint64_t n_nonedge;
    uint64_t n_uncovered;
    uint64_t n_pairs_bad;
    uint64_t first_bad_vertex;
    uint64_t first_uncovered;
} mm_verdict;

/* Library version string, e.g. "skipper-gb300 0.1 sm_103a". */
const char *mm_version(void);

/* Message of the last failing call on this thread ("" if none). */
const char *mm_last_error(void);

/* Fill *o with the defaults.  Returns MM_ERR_ARG when o is NULL. */
mm_status mm_default_options(mm_options *o);

/*
 * Create a handle over a device CSR (Section II-A).  Borrows d_offsets
 * (int64_t[n+1]) and d_nbrs (uint32_t[nnz], 16-byte aligned); allocates the
 * state array (ceil(n/4) words), the merge-path partition table and control
 * words on the current device.  With MM_CHECK_CSR the CSR is checked on the
 * device before returning (offsets[0] = 0, non-decreasing, offsets[n] = nnz,
 * every id < n) and MM_ERR_BAD_GRAPH is returned on failure.
 * MM_BATCH_LOCAL_IDS: the CSR is a batch packed for mm_skipper_batched whose
 * member graphs keep local ids; n (the batch's vertices) may be up to
 * MM_MAX_BATCH_VERTICES.  Such a handle runs mm_skipper_batched,
 * mm_autotune_batched and mm_validate_batched only (the other calls return
 * MM_ERR_UNSUPPORTED), and MM_CHECK_CSR and MM_HOST_MAPPED are not available
 * with it (MM_ERR_UNSUPPORTED).
 * Errors: MM_ERR_ARG (null out, n > MM_MAX_VERTICES, null arrays with n or
 * nnz > 0, misaligned d_nbrs), MM_ERR_OOM, MM_ERR_CUDA, MM_ERR_BAD_GRAPH,
 * MM_ERR_UNSUPPORTED.
 */
#define MM_MAX_BATCH_VERTICES (1ull << 40)
mm_status mm_create_csr(uint64_t n, uint64_t nnz, const int64_t *d_offsets,
                        const uint32_t *d_nbrs, uint32_t flags, void *cuda_stream,
                        mm_graph **out);
/*
 * MM_HOST_MAPPED (mm_create_csr and mm_create_coo): the input arrays are host
 * addresses -- page-locked memory (cudaHostAlloc, cudaHostRegister, a pinned
 * torch tensor), or, on a device that reads pageable memory through the
 * host's page tables (Grace-Blackwell), any host memory.  The handle takes
 * their device addresses (cudaHostGetDevicePointer) and every kernel reads
 * them in place through the host link -- NVLink-C2C on a Grace-Blackwell
 * node -- so a call moves only what it reads: the sweep's row skip leaves
 * most neighbour ids of a dense graph unread, which a copy of the whole CSR
 * would move all the same, and on such a handle the sweep loads ids
 * selectively by default (mm_options.id_loads).  The state array, the mate output and all scratch
 * stay in device memory.  The arrays must stay valid and unchanged while the
 * handle is used.  MM_ERR_ARG when the device cannot address an array.
 */

/*
 * Create a handle over an edge list in coordinate form (Section V-C: Skipper
 * may read its input as a list of edges, with no symmetrisation).  Edge i is
 * {d_src[i], d_dst[i]}; each undirected edge needs to be listed once, in
 * either direction, in any order; repeats and self-loops are allowed (a
 * repeat is resolved at once by the line-10 test, a loop is skipped).
 *   d_src, d_dst  uint32_t[m] in device memory, borrowed, 4-byte aligned
 *                 (16-byte aligned for 128-bit loads; otherwise 32-bit loads).
 * The handle owns its state array and control words, as for a CSR.  With
 * MM_CHECK_CSR every id is checked (< n) on the device before returning.
 * mm_skipper on this handle runs Algorithm 1 for every listed edge (there is
 * no row, so none is skipped; o->grain counts edges per work unit); serial
 * mode takes the edges in list order and equals sequential greedy over the
 * list.  mm_validate checks against the listed edges (first_uncovered is a
 * list index); mm_get_stats counts 128-edge tiles as chunks.  The batched
 * calls reject this handle with MM_ERR_UNSUPPORTED.
 * Errors: MM_ERR_ARG (null out, n > MM_MAX_VERTICES, null arrays with m > 0,
 * misaligned arrays, unknown flags), MM_ERR_OOM, MM_ERR_CUDA, MM_ERR_BAD_GRAPH.
 */
mm_status mm_create_coo(uint64_t n, uint64_t m, const uint32_t *d_src, const uint32_t *d_dst,
                        uint32_t flags, void *cuda_stream, mm_graph **out);

/*
 * The device address of host memory that kernels can read in place: the
 * lookup MM_HOST_MAPPED makes (page-locked memory, or any host memory on a
 * device that walks the host's page tables), for callers who fill
 * mm_graph_desc entries themselves.  Writes it to *device_out.  No paper
 * counterpart: it exists for the host-resident inputs of this library.
 * Errors: MM_ERR_ARG (null argument, or memory the device cannot address).
 */
mm_status mm_host_device_address(const void *host, const void **device_out);

/*
 * Skipper's single pass (Algorithm 1): every vertex starts ACC (lines 3-4);
 * every stored entry (x, y), x != y, is resolved once with u = min(x, y),
 * v = max(x, y): reserve u ACC->RSVD, claim v ACC->MCHD, then set u MCHD or
 * release it to ACC (lines 5-18).  Entries are split into equal merge-path
 * units over rows and entries (the GPU form of the paper's equal-edge blocks,
 * Section IV-C); once the row vertex x is MCHD the rest of row x is not read.
 *
 *   d_mate   uint32_t[n], caller-owned, written in full.
 *   d_pairs  uint32_t[2*cap] or NULL: pairs (u, mate[u]), u < mate[u], ascending u.
 *   d_count  uint64_t[1] or NULL: number of pairs (written when d_pairs or
 *            d_count is given; pairs beyond cap are counted, not written).
 * Waits for the GPU unless o->nosync; returns MM_ERR_TIMEOUT when a wait ran
 * past o->spin_limit, MM_ERR_BAD_GRAPH when an id >= n was met.  The result
 * is a maximal matching; which one depends on timing (Section V-C), except in
 * serial mode, where it is the sequential greedy result.
 */
mm_status mm_skipper(mm_graph *g, const mm_options *o, uint32_t *d_mate, uint32_t *d_pairs,
                     uint64_t cap, uint64_t *d_count, void *cuda_stream);

/*
 * The same pass (Algorithm 1) with its result copied into host memory while
 * it runs.  The merge-path units are taken in ascending order, in `pieces`
 * consecutive launches of about equal unit counts; once a launch has ended,
 * every row before the first row of the next unit has been walked to its end,
 * so each of those vertices is MCHD or has only MCHD neighbours (Section
 * II-B's maximality, row by row) and its mate can no longer change.  That
 * prefix of d_mate is copied to h_mate on a second stream while the next
 * launches run; the last copy follows the last launch.  No paper
 * counterpart: it hides the device-to-host copy of the result behind the pass
 * for callers whose results go to host memory.
 *
 *   d_mate   uint32_t[n] in device memory, caller-owned, written in full.
 *   h_mate   uint32_t[n] in page-locked host memory, caller-owned, equal to
 *            d_mate when the call has completed.
 *   pieces   1..MM_MAX_PIECES launches (fewer when the graph has fewer units).
 * o as for mm_skipper, with units in ascending order (MM_ORDER_AUTO is taken
 * as ascending; MM_ORDER_DISPERSED, serial, stats, timing and use_graph give
 * MM_ERR_UNSUPPORTED).  Edge-list and MM_BATCH_LOCAL_IDS handles:
 * MM_ERR_UNSUPPORTED.  Errors: MM_ERR_ARG (null arrays with n > 0, pieces out
 * of range, h_mate not page-locked host memory), MM_ERR_TIMEOUT,
 * MM_ERR_BAD_GRAPH, MM_ERR_CUDA.  Waits for the GPU (after one short wait
 * for the prepare step, whose partition sets the copies' sizes) unless
 * o->nosync, in which case mm_sync or a wait on the stream ends the call.
 */
#define MM_MAX_PIECES 64u
mm_status mm_skipper_to_host(mm_graph *g, const mm_options *o, uint32_t *d_mate, uint32_t *h_mate,
                             uint32_t pieces, void *cuda_stream);

/*
 * Batched Skipper over num_graphs graphs packed block-diagonally in the
 * handle's CSR: graph k owns vertices [vbase[k], vbase[k+1]) and entries
 * [ebase[k], ebase[k+1]), and no entry leaves its block.  One persistent sweep
 * covers all graphs (Skipper on the union is Skipper on each block, since no
 * edge crosses blocks).  d_vbase, d_ebase: int64_t[num_graphs+1] in device
 * memory, vbase[0] = ebase[0] = 0, vbase[num_graphs] = n, ebase[num_graphs] =
 * nnz, non-decreasing.  d_mate: uint32_t[n].  d_graph_pairs: uint64_t[num_graphs]
 * or NULL, matched pairs per graph.
 *
 * Ids.  On a handle made without MM_BATCH_LOCAL_IDS the neighbour ids and the
 * mate entries are global (vertex x of graph k is vbase[k] + x).  On a handle
 * made with MM_BATCH_LOCAL_IDS they are local: graph k's entries hold ids in
 * [0, vbase[k+1] - vbase[k]), and d_mate[vbase[k] + x] receives the local id of
 * x's partner; the offsets stay global entry indices.  The batch's total n may
 * then exceed MM_MAX_VERTICES (each graph's n may not).
 *
 * Work split.  Without a cap (warps_per_graph = 0) on a global-id handle, the
 * union is split into merge-path units of `grain` rows + entries (units may
 * span graphs).  With local ids or warps_per_graph > 0, every graph is split
 * on its own into min(warps_per_graph, ceil(items / grain)) units (no cap when
 * 0); those tables are computed on the device from d_vbase / d_ebase at every
 * call.  With o->serial each graph is walked by one thread in SGMM order (the
 * result equals sequential greedy MM on every graph).  With o->use_graph the
 * launches run as a CUDA graph built once per handle and option set, whose
 * kernel arguments are updated per call (new buffers or contents need no new
 * graph).  stats and poison_vertex are not available with local ids or a cap
 * (MM_ERR_UNSUPPORTED).
 */
mm_status mm_skipper_batched(mm_graph *g, uint64_t num_graphs, const int64_t *d_vbase,
                             const int64_t *d_ebase, const mm_options *o, uint32_t *d_mate,
                             uint64_t *d_graph_pairs, void *cuda_stream);

/*
 * The exact checker (Section II-B) over a batch laid out as for
 * mm_skipper_batched, global or local ids as the handle says: every member
 * graph is checked on its own vertices and entries and the counts are summed
 * into one verdict.  first_bad_vertex is a batch vertex index (vbase[k] + x),
 * first_uncovered a batch entry index.  On a global-id handle the verdict
 * equals mm_validate's.  Synchronous.  Errors: MM_ERR_ARG, MM_ERR_CUDA,
 * MM_ERR_OOM.
 */
mm_status mm_validate_batched(mm_graph *g, uint64_t num_graphs, const int64_t *d_vbase,
                              const int64_t *d_ebase, const uint32_t *d_mate, mm_verdict *h_out,
                              void *cuda_stream);

/*
 * Exact checker on the device (Section II-B; counting rules above).
 * d_pairs may be NULL (count ignored).  Synchronous: *h_out is filled before
 * return.  Errors: MM_ERR_ARG, MM_ERR_CUDA, MM_ERR_OOM.
 */
mm_status mm_validate(mm_graph *g, const uint32_t *d_mate, const uint32_t *d_pairs,
                      uint64_t count, mm_verdict *h_out, void *cuda_stream);

/* Wait for the handle's last call on cuda_stream and return its device status
 * (MM_OK, MM_ERR_TIMEOUT or MM_ERR_BAD_GRAPH).  Used after nosync calls. */
mm_status mm_sync(mm_graph *g, void *cuda_stream);

/* Statistics of the last mm_skipper call made with o->stats = 1 (waits for it).
 * MM_ERR_ARG when no such call was made. */
mm_status mm_get_stats(mm_graph *g, mm_stats *out, void *cuda_stream);

/* Debugging aid: counts of the states the last mm_skipper call on g left in
 * its state array (the handle's packed states, or the mate array itself in
 * the 32-bit layout): out[0] ACC, out[1] RSVD, out[2] MCHD, out[3] any other
 * field value (never produced).  After a completed call RSVD is 0 and MCHD is
 * twice the matched pairs (Fig. 4: every reservation ends in MCHD or ACC).
 * Synchronous.  MM_ERR_ARG when no mm_skipper call was made on g. */
mm_status mm_state_census(mm_graph *g, uint64_t out[4], void *cuda_stream);

/* Per-kernel times of the last call made with o->timing = 1 (waits for its
 * events).  MM_ERR_ARG when no timed call was made since the last
 * mm_timing_history. */
mm_status mm_get_timing(mm_graph *g, mm_timing *out);

/* Per-kernel times of the latest timed calls (at most 256 are kept), oldest
 * first: writes min(max, kept) entries to out[], their number to *count, and
 * clears the history.  Timed calls record CUDA events on their stream and do
 * not wait for them; this call waits. */
mm_status mm_timing_history(mm_graph *g, mm_timing *out, uint32_t max, uint32_t *count);

/*
 * Autotuner for mm_skipper on one handle: times the candidate settings --
 * grain in {2048, 8192}, status_bits in {2, 8, 32}, block_threads 512 with
 * blocks_per_sm either the 40-register or the 32-register instance's
 * occupancy, unit_order ascending or dispersed (edge-list handles: grain and
 * status_bits only) -- on this graph with CUDA events: one untimed and three
 * timed runs each, a candidate whose first timed run is already 1.5x slower
 * than the best run so far being dropped.  Every new best is checked by
 * mm_validate (an invalid result fails the call with MM_ERR_CUDA), and the
 * fastest is written into *o; other fields of *o (symmetric, id_loads, ...)
 * are kept and apply to every candidate.  d_mate_scratch: uint32_t[n].
 * Synchronous.  No paper counterpart (the paper has no tuning parameters;
 * the GPU's state width, occupancy and unit order are this library's).
 * Errors: MM_ERR_ARG, MM_ERR_UNSUPPORTED (a MM_BATCH_LOCAL_IDS handle), and
 * those of mm_skipper.
 */
mm_status mm_autotune(mm_graph *g, uint32_t *d_mate_scratch, mm_options *o, void *cuda_stream);

/*
 * Autotuner for mm_skipper_batched: times the candidate settings -- grain in
 * {1024, 2048, 4096, 8192}, status_bits in {2, 8, 32}, block_threads 512 with
 * blocks_per_sm either the 40-register instance's or the 32-register
 * instance's occupancy (see blocks_per_sm), unit_order ascending or dispersed,
 * warps_per_graph in {0 (no cap), 4, 16} -- on this batch with CUDA
 * events: one untimed and three timed runs each, a candidate whose first timed
 * run is already 1.5x slower than the best run so far being dropped.  Every
 * new best is checked by the device checker (mm_validate_batched; an invalid
 * result fails the call with MM_ERR_CUDA), and the fastest is written into
 * *o (other fields of *o are kept).  d_mate_scratch: uint32_t[n].
 * Synchronous.
 */
mm_status mm_autotune_batched(mm_graph *g, uint64_t num_graphs, const int64_t *d_vbase,
                              const int64_t *d_ebase, uint32_t *d_mate_scratch,
                              mm_options *o, void *cuda_stream);

/*
 * Many independent graphs, each in its own device buffers, in one persistent
 * launch -- the form a request server uses: requests keep their CSR resident
 * where it was copied, and every graph admitted since the last launch is
 * matched together (no repacking).  Each graph is split into merge-path units
 * of `grain` rows + entries like a single graph (Section IV-C's equal-edge
 * blocks); the units of all graphs are handed out from one counter.
 *
 * mm_graph_desc: n, nnz, offsets int64_t[n+1], nbrs uint32_t[nnz] (16-byte
 * aligned) and mate uint32_t[n], all in device memory and owned by the
 * caller; with status_bits 32 mate is also the graph's state array, with 8
 * the handle keeps one state byte per vertex for all graphs.
 *
 * mm_multi_create: a handle that owns the device tables, partition, state
 * pool, checker counters and control words; it grows them (cudaMalloc) only
 * when a call needs more than any earlier call.  Calls on one handle must be
 * ordered (one stream, or synchronised by the caller).
 * mm_skipper_multi: options as mm_skipper (status_bits, serial -- one thread
 * per graph in SGMM order --, grain, block_threads, blocks_per_sm, spin_limit,
 * nosync); timing, use_graph, poison_vertex and l2_persist give
 * MM_ERR_UNSUPPORTED.  Waits for the GPU unless nosync (then mm_multi_sync).
 * mm_validate_multi: the exact checker (counting rules above, without a pair
 * list) for every graph at once; h_out[k] is graph k's verdict.  Synchronous.
 * mm_validate_multi_async enqueues the same check on the stream (it may follow
 * an mm_skipper_multi call on the same stream at once: the two use separate
 * tables); once the stream has passed it, mm_multi_verdicts writes the
 * verdicts of that check (num_graphs must match).
 */
typedef struct mm_graph_desc {
    uint64_t n;
    uint64_t nnz;
    const int64_t *offsets;
    const uint32_t *nbrs;
    uint32_t *mate;
} mm_graph_desc;

typedef struct mm_multi mm_multi;

mm_status mm_multi_create(mm_multi **out);
mm_status mm_skipper_multi(mm_multi *m, uint64_t num_graphs, const mm_graph_desc *h_descs,
                           const mm_options *o, void *cuda_stream);
mm_status mm_multi_sync(mm_multi *m, void *cuda_stream);
mm_status mm_validate_multi(mm_multi *m, uint64_t num_graphs, const mm_graph_desc *h_descs,
                            mm_verdict *h_out, void *cuda_stream);
mm_status mm_validate_multi_async(mm_multi *m, uint64_t num_graphs, const mm_graph_desc *h_descs,
                                  void *cuda_stream);
mm_status mm_multi_verdicts(mm_multi *m, uint64_t num_graphs, mm_verdict *h_out);
mm_status mm_multi_destroy(mm_multi *m);

/* Release the handle's scratch.  Does not touch the borrowed CSR. */
mm_status mm_destroy(mm_graph *g);

/*
 * mm_skipper_static -- the same matching pass as mm_skipper, for callers that
 * cannot allocate device memory while they run (a program whose device memory
 * all belongs to its own pool after start-up, a serving loop that must not
 * allocate per request, a plug-in inside a process whose allocator it does not
 * own).  The paper has no counterpart to this call.
 *
 * No handle and no cudaMalloc: the pass keeps its scratch (one state byte per
 * vertex, the merge-path partition table, the work counter and error word) in
 * one fixed 8 MiB device array inside the library, which every GPU that loads
 * the library holds until the process exits.  The caller passes the device CSR
 * (same layout and alignment rules as mm_create_csr; it is not checked) and
 * the mate array d_mate (uint32_t[n], written in full).
 *
 * Limits: n <= MM_STATIC_MAX_VERTICES (larger graphs return MM_ERR_ARG, with
 * the reason in mm_last_error()); the grain is raised when needed so that the
 * partition fits the fixed table.  Options: status_bits 0 or 8, serial, grain,
 * block_threads, blocks_per_sm, spin_limit, poison_vertex, id_loads AUTO or
 * EAGER, unit_order; blocks_per_sm 0 and MM_ORDER_AUTO follow mm_options'
 * rule for the byte state array.  The options that need a handle's own
 * memory -- timing, use_graph, nosync, l2_persist, stats, stage_windows, symmetric and id_loads SELECTIVE
 * -- give MM_ERR_UNSUPPORTED; nothing is ignored silently.  The call waits for
 * its work and returns MM_OK, MM_ERR_TIMEOUT, MM_ERR_BAD_GRAPH, MM_ERR_ARG,
 * MM_ERR_UNSUPPORTED or MM_ERR_CUDA, with the reason of every failure in
 * mm_last_error().
 *
 * Every call looks up the array's address in the calling thread's current
 * context, so the call stays correct after cudaDeviceReset and in a context
 * that is not the device's primary one (each context holds its own copy of
 * the array).  The first call in a context loads the library's device code
 * there: make it before any stream capture.  All calls in one context share
 * the one array: each call clears what must start at zero, and calls whose
 * work overlaps on the GPU (two host threads, two streams) race on it and must
 * be serialised by the caller.
 */
#define MM_STATIC_MAX_VERTICES 7864064ull
mm_status mm_skipper_static(uint64_t n, uint64_t nnz, const int64_t *d_offsets,
                            const uint32_t *d_nbrs, uint32_t *d_mate, const mm_options *o,
                            void *cuda_stream);

/* ------------------------------------------------------------------------
 * Serving: a continuous-batching server over graphs that live in host memory.
 * No paper counterpart (the paper runs one graph at a time); it serves many
 * independent requests through the multi-graph pass above.
 *
 * One worker thread admits requests in arrival order (no overtaking) while
 * their device footprint fits memory_bytes and, whenever a compute slot is
 * free, launches one mm_skipper_multi pass over everything admitted since the
 * last launch, followed on the same stream by mm_validate_multi_async when
 * validate is set.  With two slots a new batch is admitted and launched while
 * the previous one runs.  A request with nnz <= in_place_max_nnz whose arrays
 * the device can address (see MM_HOST_MAPPED) is read in place and its mate
 * lives in a per-launch device arena; any other request is copied to its own
 * stream-ordered device buffers.  Each mate array is copied back into the
 * caller's h_mate_out.  The caller's arrays must stay valid and unchanged
 * until the request's result has been collected.
 * ------------------------------------------------------------------------ */
typedef struct mm_server mm_server;

typedef struct mm_server_config {
    uint64_t memory_bytes;        /* device bytes resident requests may hold; 0 = the
                                     free memory at creation minus reserve_bytes */
    uint64_t reserve_bytes;       /* default 8 GiB */
    uint64_t max_graphs_per_tick; /* graphs per launch, default 4096 */
    uint64_t max_bytes_per_tick;  /* device bytes admitted per launch, default 32 GiB
                                     (one larger request runs alone) */
    uint64_t in_place_max_nnz;    /* largest request read in place, default 1 << 20 */
    uint32_t validate;            /* 1 (default): check every result before completion */
    uint32_t slots;               /* compute slots, 1 or 2 (default) */
    mm_options opts;              /* options of the pass (status_bits, grain, serial, ...) */
    uint64_t reserved[4];
} mm_server_config;

typedef struct mm_server_result {
    mm_status status;    /* MM_OK; the pass's failure (MM_ERR_TIMEOUT, MM_ERR_BAD_GRAPH);
                            MM_ERR_OOM when the request can never fit memory_bytes;
                            MM_ERR_CUDA and the like when the server failed */
    uint32_t in_place;   /* 1 when the request was read in place */
    mm_verdict verdict;  /* the checker's verdict (validate set, status MM_OK) */
    int64_t submit_ns;   /* CLOCK_MONOTONIC at submission */
    int64_t done_ns;     /* CLOCK_MONOTONIC when the mate and the verdict were ready */
} mm_server_result;

/* Defaults (above) into *c.  MM_ERR_ARG for a null pointer. */
mm_status mm_server_default_config(mm_server_config *c);
/* Start a server on the current device.  MM_ERR_ARG (bad config), MM_ERR_CUDA,
 * MM_ERR_OOM. */
mm_status mm_server_create(const mm_server_config *c, mm_server **out);
/* Queue one graph: host CSR (n vertices, nnz entries) and an n-entry host
 * output h_mate_out (page-locked for an asynchronous copy).  Writes the
 * request's ticket.  Thread-safe.  MM_ERR_ARG on a null array, n too large,
 * or a closing server; the server's failure status once it has failed. */
mm_status mm_server_submit(mm_server *s, uint64_t n, uint64_t nnz, const int64_t *h_offsets,
                           const uint32_t *h_nbrs, uint32_t *h_mate_out, uint64_t *ticket);
/* Collect a request's result, waiting up to timeout_s seconds (0 = poll).
 * MM_OK with *out filled (each result is collected once), or MM_PENDING. */
mm_status mm_server_wait(mm_server *s, uint64_t ticket, double timeout_s, mm_server_result *out);
/* Launches so far, graphs launched, device bytes held by admitted requests
 * (any pointer may be NULL). */
mm_status mm_server_stats(mm_server *s, uint64_t *launches, uint64_t *graphs,
                          uint64_t *device_bytes_held);
/* Drain every queued request, then release the server.  Results not yet
 * collected are dropped.  Returns the server's failure status, if any. */
mm_status mm_server_destroy(mm_server *s);
/* Admission arithmetic, exposed for tests: the device bytes a request holds
 * while resident (in place: mate and scratch; copied: plus its CSR), and how
 * many of the pending sizes (arrival order) fit: stops at the first that does
 * not (no overtaking) or at max_graphs. */
mm_status mm_server_device_bytes(uint64_t n, uint64_t nnz, uint32_t in_place, uint64_t *out);
mm_status mm_server_plan_admission(const uint64_t *sizes, uint64_t count, uint64_t used,
                                   uint64_t budget, uint64_t max_graphs, uint64_t *k_out,
                                   uint64_t *bytes_out);

#ifdef __cplusplus
}
#endif

#endif /* SKIPPER_H */
