/*
 * tectonic.h -- C ABI of the GB300 (sm_103a) motif-based community detection
 * library (Chen & Tsourakakis, "Parallel Motif-Based Community Detection",
 * arXiv 2412.12382).
 *
 * The library runs Algorithm 1 of the paper on one GPU: per-edge triangle
 * counts t(u,v) and wedge counts (Sec. I, "Notations"), the Tectonic and TW
 * similarities (Table 1, Eq. 1), pruning of every edge whose similarity is
 * below a rational threshold delta = p/q, and the connected components of what
 * is left.  Components are also computed for many thresholds at once.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - Every call returns a tec_status; TEC_OK is 0.  tec_last_error() gives a
 *   human-readable message for the calling thread's last failure.  No C++
 *   exception crosses this interface.
 * - Graphs: undirected, simple (no self-loops, no duplicate edges), stored as a
 *   symmetric CSR with both directions of every edge, rows sorted ascending,
 *   vertices 0..n-1 (n < 2^31), row offsets int32 or int64, column ids int32.
 *   m = nnz / 2 undirected edges.
 * - Canonical edge order: edge e in [0, m) is the e-th pair (u, v), u < v, in
 *   lexicographic order, i.e. the upper-triangle entries of the CSR row by
 *   row.  Every per-edge output (t, wedge, weights, keep mask) uses it.
 * - Pointers are DEVICE pointers unless a flag or the parameter's description
 *   says host.  Outputs go into caller-allocated buffers of the documented
 *   size; the library never frees caller memory.
 * - A tec_graph owns a copy of the input CSR and all of its own scratch; the
 *   caller may free its input buffers as soon as tec_graph_load returns.
 *   Internal memory is released by tec_graph_free.
 * - Work is issued asynchronously on the graph's CUDA stream (a cudaStream_t
 *   passed as void*; NULL is the legacy default stream).  A call that returns
 *   a host scalar (kept count, number of components) waits for that stream.
 *   Device-side failures (a capped loop that ran out, an invalid CSR found by
 *   validation) are recorded in a device status word and reported by the next
 *   call that waits, or by tec_sync.
 * - A tec_graph is not thread-safe: one host thread at a time per graph.
 */
#ifndef TECTONIC_H
#define TECTONIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tec_status {
    TEC_OK = 0,
    TEC_EINVAL = 1,     /* a bad argument (NULL pointer, size out of range, q <= 0) */
    TEC_ENOMEM = 2,     /* a device or host allocation failed */
    TEC_ECUDA = 3,      /* a CUDA runtime call failed; the message names it */
    TEC_ETIMEOUT = 4,   /* a bounded device loop hit its cap; the graph stays usable */
    TEC_EOVERFLOW = 5,  /* a size or threshold does not fit the checked integer width */
    TEC_EBADGRAPH = 6,  /* validation found an unsorted row, self-loop, duplicate or asymmetry,
                           or a label or block id was out of range */
    TEC_ESTATE = 7,     /* a call needs a step that has not been run (e.g. components before prune) */
    TEC_EIO = 8         /* a checkpoint file could not be opened, read or written, or is not a valid
                           picker checkpoint (wrong magic, version, shape, size or checksum) */
} tec_status;

/* Similarity functions of Table 1. */
typedef enum tec_measure {
    TEC_TECTONIC = 0,   /* t(u,v) / (deg u + deg v) */
    TEC_TW = 1,         /* t(u,v) - wedge(u,v) = 3 t(u,v) + 2 - deg u - deg v (Eq. 1) */
    TEC_JACCARD = 2,    /* t(u,v) / |N(u) u N(v)| = t / (deg u + deg v - t) (Sec. II, Proposition 1) */
    TEC_K3 = 3,         /* t(u,v), the edge's triangle count */
    TEC_K4 = 4          /* K4(u,v), the 4-cliques containing the edge (saturating at 2^32 - 1;
                           thresholds above 2^32 - 1 are TEC_EOVERFLOW) */
} tec_measure;

/* tec_graph_load flags */
#define TEC_HOST_PTR 0x1u   /* row_off / col are host pointers (pinned or pageable) */
#define TEC_VALIDATE 0x2u   /* check the CSR invariants on the device; TEC_EBADGRAPH if violated */

typedef struct tec_graph tec_graph;

/* Library version as 10000*major + 100*minor + patch. */
int tec_version(void);

/* Copies the calling thread's last error message (NUL-terminated, truncated to
 * len) into buf and returns its full length.  buf may be NULL when len is 0. */
size_t tec_last_error(char *buf, size_t len);

/* ---------------------------------------------------------------- graphs */

/* Creates an empty graph with room for n_cap vertices and nnz_cap CSR entries
 * (2 x undirected edges), allocating all device memory a pass needs on the
 * current CUDA device.  stream: cudaStream_t (void*) that every later call on
 * this graph uses.  TEC_ENOMEM if the device lacks memory. */
tec_status tec_graph_create(int64_t n_cap, int64_t nnz_cap, void *stream, tec_graph **out);

/* Loads a symmetric CSR (n vertices, nnz = 2m entries) into g, replacing any
 * previous graph and its results.  row_off: n+1 offsets, int64 if off_is_i64
 * else int32; col: nnz int32 ids.  flags: TEC_HOST_PTR, TEC_VALIDATE.
 * TEC_EINVAL if n > n_cap or nnz > nnz_cap; TEC_EBADGRAPH under TEC_VALIDATE
 * (waits for the stream).  Vertex degrees deg(u) = row lengths are computed
 * here. */
tec_status tec_graph_load(tec_graph *g, const void *row_off, int off_is_i64, const int32_t *col,
                          int64_t n, int64_t nnz, uint32_t flags);

/* tec_graph_create with exactly the needed capacity, then tec_graph_load. */
tec_status tec_graph_upload(const void *row_off, int off_is_i64, const int32_t *col, int64_t n,
                            int64_t nnz, uint32_t flags, void *stream, tec_graph **out);

/* Waits for the graph's stream, frees every internal buffer and the handle. */
tec_status tec_graph_free(tec_graph *g);

/* Host scalars: vertex count and undirected edge count of the loaded graph. */
tec_status tec_graph_info(const tec_graph *g, int64_t *n, int64_t *m);

/* Waits for the graph's stream and reports any device-side failure recorded
 * since the last wait (TEC_ETIMEOUT, TEC_EBADGRAPH), clearing it. */
tec_status tec_sync(tec_graph *g);

/* ---------------------------------------------------------------- steps */

/* Degree-ordered orientation (Sec. II cites Shun & Tangwongsan for ranking by
 * degree): keeps u -> v iff (deg u, u) < (deg v, v), so each undirected edge
 * is stored once and every out-row stays sorted.  Needed by every later step;
 * the steps below run it themselves when it has not been run. */
tec_status tec_orient(tec_graph *g);

/* Per-edge triangle counts t(u,v) = |N(u) n N(v)| (Sec. I) for all m edges,
 * kept on the device for the steps below (Sec. III-C computes the same
 * quantity by one merge per edge; here every triangle is listed once from its
 * lowest-ranked vertex and credited to its three edges). */
tec_status tec_support(tec_graph *g);

/* Canonical edge list: u_out[e] < v_out[e], m entries each (device). */
tec_status tec_edge_list(tec_graph *g, int32_t *u_out, int32_t *v_out);

/* t(u,v) into t_out[m] and, if wedge_out is not NULL,
 * wedge(u,v) = |N(u) u N(v)| - t(u,v) - 2 = deg u + deg v - 2 t(u,v) - 2
 * into wedge_out[m] (Sec. I), both uint32 in canonical order (device). */
tec_status tec_edge_support(tec_graph *g, uint32_t *t_out, uint32_t *wedge_out);

/* K4 participation (Table 1, kappa = 4): for every edge, the number of
 * 4-cliques containing it, i.e. the edges {c, d} inside the common
 * neighbourhood N(u) n N(v).  k4_out: device, m uint32 in canonical order,
 * saturating at 2^32 - 1.  Runs tec_support if needed; the counts are kept for
 * TEC_K4 pruning until the triangle counts are recomputed. */
tec_status tec_edge_k4(tec_graph *g, uint32_t *k4_out);

/* Similarity of every edge as float64 in canonical order (device):
 * TEC_TECTONIC: t / (deg u + deg v), one correctly rounded IEEE division;
 * TEC_TW: t - wedge, an integer, exactly representable;
 * TEC_JACCARD: t / (deg u + deg v - t), one correctly rounded IEEE division;
 * TEC_K3: t, exactly representable;
 * TEC_K4: the K4 participation count (tec_edge_k4), exactly representable. */
tec_status tec_edge_weights(tec_graph *g, tec_measure measure, double *w_out);

/* Algorithm 1, first step: keeps edge e iff sim(e) >= p/q, i.e. removes
 * exactly the edges with sim(e) < delta.  Decided in exact integer arithmetic
 * (64-bit products when |p|, q < 2^28, 128-bit otherwise):
 *   Tectonic: t*q >= p*(deg u + deg v);   TW: (3t + 2 - deg u - deg v)*q >= p;
 *   Jaccard:  t*q >= p*(deg u + deg v - t);   K3: t*q >= p;   K4: K4(e)*q >= p.
 * q must be > 0 (TEC_EINVAL); |p| and q must be < 2^62, and a K4 threshold
 * at most 2^32 - 1 (TEC_EOVERFLOW).
 * keep_out (device, m bytes, canonical order) may be NULL; kept_out (HOST,
 * may be NULL; waits when given) receives the number of kept edges.  The mask
 * stays on the device for tec_components. */
tec_status tec_prune(tec_graph *g, tec_measure measure, int64_t p, int64_t q, uint8_t *keep_out,
                     int64_t *kept_out);

/* Algorithm 1, second step: connected components of (V, kept edges) of the
 * last tec_prune.  labels_out (device, n int32): the smallest vertex id of each
 * vertex's component (an isolated vertex is its own label).  ncomp_out (HOST,
 * may be NULL; waits when given): number of components.  TEC_ESTATE if no
 * prune has run. */
tec_status tec_components(tec_graph *g, int32_t *labels_out, int64_t *ncomp_out);

/* Algorithm 1 repeated for k thresholds delta_i = p[i]/q[i], as the paper
 * does when it sweeps delta (Sec. IV-D, Fig. 6; Table 4's TW grid), in one
 * call.  Components at k thresholds at once: for each threshold i, the labels (and
 * number of components) that tec_prune(p[i], q[i]) + tec_components would give,
 * through a maximum spanning forest of the edge levels (the number of
 * thresholds each edge survives) and one offline union-find sweep over the
 * forest edges, highest level first.  Thresholds may come in any order and
 * may repeat; 1 <= k <= 127; p, q are HOST arrays.  labels_out (device,
 * k x n int32, row i for threshold i).  A batch of graphs is loaded as one
 * disjoint union: seg_off (device, nseg+1 int64 vertex offsets of the graphs,
 * or NULL) makes every label relative to its graph's first vertex, and
 * ncomp_out (HOST, may be NULL; waits) receives k x nseg component counts (k
 * counts without segments).  This segment table is the batch interface: a
 * batch of many graphs (for example the 256 degree-corrected SBM graphs of
 * one sweep launch) is tec_graph_load of their disjoint union plus seg_off,
 * so no separate batch upload or batch sweep call is needed.  Replaces the last prune's mask state.  Without
 * ncomp_out the call does not wait: device-side errors (a forest still
 * growing after ceil(log2 n) + 2 Boruvka rounds, TEC_ETIMEOUT; a malformed
 * forest, TEC_EBADGRAPH) are reported by the next call that waits.  Once a
 * first call has allocated the sweep's buffers (and the triangle counts
 * exist), a call without ncomp_out issues only kernels and memsets on the
 * graph's stream and can be captured in a CUDA graph. */
tec_status tec_sweep(tec_graph *g, tec_measure measure, const int64_t *p, const int64_t *q, int k,
                     const int64_t *seg_off, int nseg, int32_t *labels_out, int64_t *ncomp_out);

/* Picker features of every graph of a batch (the whole graph if seg_off is
 * NULL): the 64-bin histogram of Tectonic weights on the grid i/128
 * (bin = min(63, floor(128 t / (deg u + deg v)))), divided by the graph's edge
 * count m, then ln(2m/n) and ln(m).  feat_out: device, nseg x 66 float32
 * (rows of zeros for graphs without edges).  Runs tec_support if needed.  The
 * paper picks thresholds by rules of thumb (Sec. IV-D); these features feed
 * the learned picker that replaces them. */
tec_status tec_features(tec_graph *g, const int64_t *seg_off, int nseg, float *feat_out);

/* Adjusted Rand index (Hubert & Arabie 1985) between k labelings (device,
 * k x n int32, e.g. the output of tec_sweep: each label is a vertex id of its
 * graph, 0 <= label < that graph's vertex count, relative to the graph's first
 * vertex when seg_off is given) and reference blocks truth (device, n int32,
 * block ids 0..63 within each graph).  A vertex whose label or block id is
 * out of range is skipped and TEC_EBADGRAPH is reported at the next wait.
 * ari_out: device, k x nseg float64 (k values without segments).  Pair counts
 * are exact integers; the final ratio has a relative error below 1e-15.  The
 * paper evaluates with matched precision / recall (Sec. IV-A); ARI is the
 * score this project trains and rates the picker by. */
tec_status tec_ari(tec_graph *g, int k, const int32_t *labels, const int32_t *truth, const int64_t *seg_off, int nseg,
                   double *ari_out);

/* Algorithm 1 for every graph of a batch, each with its own threshold
 * p[s]/q[s] (DEVICE int64 arrays, nseg entries; an edge belongs to the graph
 * of its endpoints): pruning with fused union-find hooking, then labels
 * relative to each graph's first vertex in labels_out (device, n int32).
 * ncomp_out (HOST, nseg, may be NULL; waits): components per graph.  A
 * threshold with q <= 0 removes every edge of its graph.  Runs the triangle
 * counts if needed. */
tec_status tec_prune_components_batch(tec_graph *g, tec_measure measure, const int64_t *p, const int64_t *q,
                                      const int64_t *seg_off, int nseg, int32_t *labels_out, int64_t *ncomp_out);

/* Per-threshold statistics of a sweep, the quantities Sec. IV-D plots
 * against the threshold (Fig. 6), for every graph of a batch (the whole graph
 * if seg_off is NULL). */
typedef struct tec_sweep_stat {
    int64_t ncomp;      /* components */
    int64_t kept;       /* edges with sim >= p/q (Algorithm 1's survivors) */
    int64_t largest;    /* vertices of the largest component */
    int64_t intra;      /* edges of the input graph with both ends in one component */
    double modularity;  /* Sec. II with the components as communities:
                           (4 m intra - sum_c vol(c)^2) / (4 m^2), vol(c) the
                           degree sum of c, from exact integers; 0 if m = 0 */
} tec_sweep_stat;

/* Statistics of k labelings (device, k x n int32, labels relative to each
 * graph when seg_off is given, row i the components at p[i]/q[i]: the output
 * of tec_sweep, or of tec_prune_components_batch at those thresholds).  Each
 * label must be the smallest vertex id of its component, as those calls
 * write it: components are counted at the vertices labelled by themselves.
 * The labelings must be nested as a sweep's are (a lower threshold never
 * splits a component); `intra` is found by binary search over them.  p, q: HOST,
 * k <= 127, q > 0.  stats_out: device, k x nseg (row-major by threshold).
 * Per-graph edge counts must stay below 2^31.  Runs tec_support if needed. */
tec_status tec_sweep_stats(tec_graph *g, tec_measure measure, const int64_t *p, const int64_t *q, int k,
                           const int32_t *labels, const int64_t *seg_off, int nseg, tec_sweep_stat *stats_out);

/* The threshold rules of thumb of Sec. IV-D, per graph, from k x nseg
 * statistics (device) of thresholds p/q (HOST, as given to tec_sweep_stats):
 *   TEC_RULE_LARGEST_JUMP: visiting the thresholds in decreasing order, the
 *     one just above the largest increase of the largest component (the
 *     highest on ties); where it never increases, TEC_RULE_MODULARITY;
 *   TEC_RULE_MODULARITY: the largest modularity (the lowest threshold on ties).
 * best_out: device, nseg int32 row indices, on `stream`. */
typedef enum { TEC_RULE_LARGEST_JUMP = 0, TEC_RULE_MODULARITY = 1 } tec_rule;
tec_status tec_rule_of_thumb(const tec_sweep_stat *stats, const int64_t *p, const int64_t *q, int k, int nseg,
                             tec_rule rule, int32_t *best_out, void *stream);

/* Precision, recall and F1 of Sec. IV-A for k labelings against reference
 * blocks (same inputs as tec_ari): every found community S is matched to the
 * block C of largest Jaccard |C n S| / |C u S| (the lowest block id on ties),
 * p = |C n S| / |S|, r = |C n S| / |C|, and the three scores are the
 * size-weighted means of p, r and 2pr / (p + r).  prf_out: device,
 * k x nseg x 3 float64 (precision, recall, F1).  Precision is a ratio of exact
 * integers; recall and F1 are float64 sums (summation order unspecified). */
tec_status tec_prf(tec_graph *g, int k, const int32_t *labels, const int32_t *truth, const int64_t *seg_off, int nseg,
                   double *prf_out);

/* For each of nseg graphs, the first of k rows of ari (device, k x nseg, as
 * written by tec_ari) with the highest value: best (device, nseg int32, row
 * index) and, if not NULL, that value (device, nseg float64), on `stream`. */
tec_status tec_ari_best(const double *ari, int k, int nseg, int32_t *best, double *best_ari, void *stream);

/* Algorithm 1 end to end on the loaded graph: orientation, triangle counts,
 * similarity, pruning at p/q and components, with pruning and the union-find
 * hooking fused into one kernel.  Same outputs as tec_prune + tec_components
 * (labels_out device, ncomp_out host or NULL). */
tec_status tec_full_pass(tec_graph *g, tec_measure measure, int64_t p, int64_t q,
                         int32_t *labels_out, int64_t *ncomp_out);

/* The same pass from host memory to host memory: copies a host CSR into g
 * (within its capacity), runs tec_full_pass and copies the labels back into
 * labels_host (n int32, HOST).  Waits for completion. */
tec_status tec_full_pass_host(tec_graph *g, const int64_t *row_off_host, const int32_t *col_host,
                              int64_t n, int64_t nnz, tec_measure measure, int64_t p, int64_t q,
                              int32_t *labels_host, int64_t *ncomp_out);

/* Core staging of the triangle counts (on by default).  Vertices of degree
 * >= D, D the smallest power of two leaving at most 2^20 of them, get dense
 * codes in id order, and a copy of the oriented columns holds those codes
 * (4 bytes per edge).  Centres of degree >= D then stage their out-rows as
 * exact bitmaps over the codes: no false positives and no positive queue.
 * (A centre with an out-row of at most 256 ids takes this path only with
 * about 2^16 probes or more; below that it keeps the hashed warp visit.)
 * Disabling it frees no memory but skips the copy and stages every centre by
 * hashing; the counts are identical either way.  The next call that needs the
 * triangle counts recomputes them. */
tec_status tec_set_core_staging(tec_graph *g, int enable);

/* Probe-row tiling of the triangle counts (off by default).  Each oriented
 * edge is intersected once, from one centre, which probes the candidate's
 * out-row.  With tiling, the vertex ids are split into `groups` ranges of
 * about equal out-row volume, and every core centre (see above) with at least
 * 8 x groups candidates is visited once per range holding some of its
 * candidates, all visits of the first range first, so that the centres
 * visited together probe the rows of one range.  Measured on R-MAT scale 26
 * it is slower at every setting tried (per-visit start-up outweighs the L2
 * reuse), so the default (0) leaves it off.  groups: -1 or 0 off, 1..4095
 * that many ranges.  Needs the core staging; without the memory for its lists
 * it is skipped.  The counts are identical with any setting; the next call
 * that needs them recomputes them.  TEC_EINVAL for other values. */
tec_status tec_set_support_tiling(tec_graph *g, int groups);

/* Instrumentation: number of kernels this library has launched in this
 * process so far (all graphs, all devices). */
long long tec_launch_count(void);

/* Instrumentation: up to 5 cudaEvent_t (as void*) that tec_full_pass and
 * tec_full_pass_host record on the graph's stream before orientation, after
 * orientation, after the triangle counts, after pruning with union-find
 * hooking, and after the component labels.  count 0 turns it off.  The events
 * stay owned by the caller and must outlive their use. */
tec_status tec_set_stage_events(tec_graph *g, void *const *events, int count);

/* Introspection: copies the degree-ordered oriented CSR (running tec_orient
 * if needed) into ooff_out (device, n+1 int64) and ocol_out (device, m int32);
 * either may be NULL.  Row u lists N+(u) ascending. */
tec_status tec_oriented_csr(tec_graph *g, int64_t *ooff_out, int32_t *ocol_out);

/* ---------------------------------------------------------------- learned threshold picker */

/* The paper picks the threshold delta by rules of thumb (Sec. IV-D: the jump
 * of the largest component, else maximum modularity).  The picker replaces
 * them with a small network trained on sweeps: inputs are the tec_features
 * rows, the output y approximates b/64 for the best grid threshold b/128 (the
 * one of highest ARI), and the prediction is b = clamp(round(64 y), 1, 64).
 * Network: 66 -> 128 (ReLU) -> 128 (ReLU) -> 1, float32 parameters in one
 * vector: W1 [128 x 66] row-major, b1 [128], W2 [128 x 128], b2 [128],
 * w3 [128], b3.  Loss: mean squared error.  Optimiser: Adam with bias
 * correction. */
#define TEC_PICKER_INPUTS 66
#define TEC_PICKER_HIDDEN 128
#define TEC_PICKER_PARAMS 25217

typedef struct tec_picker tec_picker;

/* Creates a picker on the current device with the given HOST initial
 * parameters (TEC_PICKER_PARAMS floats; NULL = zeros), Adam moments zero.
 * stream: cudaStream_t (void*) used by every later call. */
tec_status tec_picker_create(const float *init_params, void *stream, tec_picker **out);
tec_status tec_picker_free(tec_picker *p);

/* Checkpointing: copies the parameters (and, if not NULL, the Adam moments
 * and the step count) to / from HOST memory.  set with NULL moments resets
 * them to zero.  Both wait. */
tec_status tec_picker_get_params(tec_picker *p, float *params_out, float *adam_m_out, float *adam_v_out,
                                 int64_t *step_out);
tec_status tec_picker_set_params(tec_picker *p, const float *params, const float *adam_m, const float *adam_v,
                                 int64_t step);

/* Checkpoint files, so that a C client can train, keep and reload a picker
 * (the parameters, both Adam moments, the step count and a free-form UTF-8
 * "meta" text such as the training record).  Format, all little-endian:
 * magic "TECPICK1"; uint32 version 1; uint32 inputs, hidden and parameter
 * counts (66, 128, 25217); int64 step; uint32 meta length L; L meta bytes;
 * then parameters, first moments and second moments, TEC_PICKER_PARAMS
 * IEEE binary32 values each; last a uint64 FNV-1a 64-bit hash of every byte
 * before it.  A file that does not match it byte for byte is TEC_EIO.
 *
 * tec_picker_file_write / _read work on HOST arrays and need no device:
 * write stores params (required), adam_m / adam_v (NULL = zeros), step and
 * meta (NUL-terminated, NULL = empty); read checks the whole file and copies
 * out what is asked for (any output may be NULL): params, moments and step,
 * up to meta_cap - 1 meta bytes plus a terminator into meta, and the full
 * meta length into *meta_len.  tec_picker_save writes a picker's current
 * state (waits for its stream); tec_picker_load creates a picker on the
 * current device (stream as in tec_picker_create) holding the file's state,
 * so training resumes where it stopped.  Not from the paper: the picker
 * replaces the rules of thumb of Sec. IV-D. */
tec_status tec_picker_file_write(const char *path, const float *params, const float *adam_m, const float *adam_v,
                                 int64_t step, const char *meta);
tec_status tec_picker_file_read(const char *path, float *params, float *adam_m, float *adam_v, int64_t *step,
                                char *meta, size_t meta_cap, size_t *meta_len);
tec_status tec_picker_save(tec_picker *p, const char *path, const char *meta);
tec_status tec_picker_load(const char *path, void *stream, tec_picker **out);

/* out[i] = network output for feats row i (device, N x 66 float32 in, N
 * float32 out).  bf16 != 0 computes every product on bfloat16 operands
 * with float32 accumulation: weights and hidden activations are rounded to
 * bfloat16, and each input is split into two bfloat16 terms (hi = bf16(x),
 * lo = bf16(x - hi)), since rounding the inputs (the log edge count, about 9
 * to 14, loses up to 0.03) would change the picked grid level far more often
 * than rounding the weights. */
tec_status tec_picker_forward(tec_picker *p, const float *feats, int64_t N, int bf16, float *out);

/* Mean squared error of the N samples (device feats N x 66, target N) into
 * *loss_out (HOST, may be NULL; waits when given) and its gradient with
 * respect to every parameter into grad_out (device, TEC_PICKER_PARAMS, may be
 * NULL).  Deterministic: batch sums run in sample order. */
tec_status tec_picker_loss_grad(tec_picker *p, const float *feats, const float *target, int64_t N, float *loss_out,
                                float *grad_out);

/* One Adam update with the given gradient (device; NULL = the gradient of the
 * last tec_picker_loss_grad). */
tec_status tec_picker_adam_step(tec_picker *p, const float *grad, float lr, float beta1, float beta2, float eps);

/* Trains for `epochs` passes over N samples (device feats / target) in
 * mini-batches of `batch`, shuffled each epoch by a keyed permutation of
 * `seed`, Adam(lr, 0.9, 0.999, 1e-8).  loss_out (HOST, epochs floats, may be
 * NULL): mean batch loss per epoch.  Waits. */
tec_status tec_picker_train(tec_picker *p, const float *feats, const float *target, int64_t N, int epochs, int batch,
                            float lr, uint64_t seed, float *loss_out);

/* The soft-level objective, for training the picker on what it is judged by.
 * ari_loss (device, N x 64 float32): row s holds, for every grid level
 * i = 1..64, the ARI that graph s loses at threshold i/128 against its best
 * level.  Per sample the loss is mix * (y - target)^2 + (1 - mix) *
 * sum_i w_i ari_loss[s][i], with w_i proportional to
 * exp(-(i - 64 y)^2 / (2 sigma^2)) and summing to 1: the expected ARI lost
 * by a level choice smoothed around 64 y (sigma in grid levels, 0.05..64;
 * mix in [0, 1]; mix = 1 is tec_picker_loss_grad's squared error).
 * tec_picker_soft_loss_grad: the mean loss (HOST, may be NULL; waits) and its
 * gradient (device, may be NULL) like tec_picker_loss_grad.
 * tec_picker_train_soft: tec_picker_train with this loss.  Not from the
 * paper: the picker replaces the rules of thumb of Sec. IV-D. */
tec_status tec_picker_soft_loss_grad(tec_picker *p, const float *feats, const float *target, const float *ari_loss,
                                     int64_t N, float sigma, float mix, float *loss_out, float *grad_out);
tec_status tec_picker_train_soft(tec_picker *p, const float *feats, const float *target, const float *ari_loss,
                                 int64_t N, int epochs, int batch, float lr, uint64_t seed, float sigma, float mix,
                                 float *loss_out);

/* The learned threshold of every graph of a batch (the whole graph if
 * seg_off is NULL): tec_features, the picker network (bf16 != 0: bfloat16
 * inference as in tec_picker_forward) and the grid threshold of
 * tec_picker_thresholds, in one call on the graph's stream (ordered after
 * work already queued on the picker's stream, and before the picker's next
 * use).  p_out, q_out: device, nseg int64 each (one without segments), ready
 * for tec_prune_components_batch.  Runs tec_support if needed.  The paper
 * picks thresholds by rules of thumb (Sec. IV-D); this call replaces them. */
tec_status tec_pick_threshold(tec_graph *g, tec_picker *p, const int64_t *seg_off, int nseg, int bf16,
                              int64_t *p_out, int64_t *q_out);

/* Grid thresholds from picker outputs y (device, N float32): b =
 * clamp(round(64 y), 1, 64) (non-finite y gives 1), p_out[i] = b,
 * q_out[i] = 128 (device int64 arrays), on `stream`. */
tec_status tec_picker_thresholds(const float *y, int64_t N, int64_t *p_out, int64_t *q_out, void *stream);

/* ---------------------------------------------------------------- no allocation */

/* Largest vertex count tec_components_noalloc accepts. */
#define TEC_NOALLOC_MAX_VERTICES 4194304

/* Connected components of an edge list, for callers that cannot allocate
 * device memory when they need the result: a host application that owns the
 * GPU memory budget, a latency-critical path that cannot pay for a
 * cudaMalloc / cudaFree (either may synchronise the device), or code that must
 * not fail for lack of memory halfway through.  The paper has no counterpart;
 * it is the union-find of tec_components with its scratch in a fixed
 * file-scope device array instead of graph-owned memory.
 *
 * n <= TEC_NOALLOC_MAX_VERTICES vertices (TEC_EINVAL beyond), m edges
 * (eu[e], ev[e]) given as device int32 arrays; keep (device, m bytes) selects
 * the edges to use, NULL uses all.  labels_out (device, n int32) receives the
 * smallest vertex id of each vertex's component; ncomp_out (host, may be NULL)
 * the number of components.  Runs on `stream`; every call then copies a
 * status word back to the host and waits for `stream`.  An endpoint outside
 * [0, n) gives TEC_EINVAL (nothing is written outside the array), and the next
 * call starts afresh.
 *
 * Allocates nothing: the union-find parents live in one device array of
 * TEC_NOALLOC_MAX_VERTICES int32 (16 MiB) that every GPU loading the library
 * holds until the process exits.  The first call on a device looks up that
 * array's device address, so make it before any stream capture.  The address
 * is kept for the life of the process: do not call this entry point on a
 * device after a cudaDeviceReset of it (the module, and with it the array, is
 * loaded anew, and the kept address is stale).  All calls on
 * a device share the array and each call re-initialises it; calls whose GPU
 * work overlaps (other streams, other host threads) race on it and must be
 * serialised by the caller. */
tec_status tec_components_noalloc(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                                  const uint8_t *keep, int32_t *labels_out, int64_t *ncomp_out,
                                  void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TECTONIC_H */
