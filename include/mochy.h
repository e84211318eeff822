/*
 * libmochy: GB300 (sm_103a) counting of hypergraph motifs (h-motifs) and
 * ternary hypergraph motifs (3h-motifs), after "Hypergraph motifs and their
 * extensions beyond binary" (arXiv 2310.15668).
 *
 * Plain C ABI.  Pointers named h_* are host memory, d_* device memory of the
 * context's GPU.  Every call returns MOCHY_OK (0) or a negative MOCHY_E_*
 * code; no exception or abort crosses the ABI.  mochy_last_error() gives a
 * one-line message for the calling thread's last failure.
 *
 * Ownership: input arrays stay owned by the caller and are copied; output
 * arrays are allocated by the caller with the stated sizes.  Device memory is
 * owned by the context and freed by mochy_destroy.  A context is used by one
 * host thread at a time.
 *
 * Limits: at most 2^26 - 1 hyperedges, 2^31 - 1 nodes, 63 nodes per
 * hyperedge; the per-hyperwedge scan kernel (exact_kernel = 1) needs at most
 * 786,432 hyperedges (it stages a row's adjacency in shared memory); the
 * split kernel keeps at most 2,096,128 rows of one hypergraph dense (the
 * tuner never picks more; a forced dense_threshold that makes more fails).
 * A call outside these limits returns MOCHY_E_UNSUPPORTED.
 *
 * Motif ids: h-motifs are numbered 1..26, 3h-motifs 1..431 (arrays are
 * indexed id-1).  The paper's figures that fix the numbering are lost; the
 * numbering used here is: canonical pattern = lexicographically smallest
 * region tuple (regions (1)..(7) of Section 2.2) over the six orders of the
 * three hyperedges; h-motifs 1-16 are closed with a non-empty triple region,
 * 17-22 open, 23-26 closed with an empty triple region, each group in
 * ascending canonical tuple order; 3h-motifs are in ascending (h-motif id,
 * canonical ternary tuple) order.  mochy_motif_pattern() returns the pattern
 * of an id.
 */
#ifndef MOCHY_H
#define MOCHY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MOCHY_OK 0
#define MOCHY_E_INVALID (-1)        /* bad argument or malformed hypergraph */
#define MOCHY_E_NOMEM (-2)          /* device allocation failed or over budget */
#define MOCHY_E_CUDA (-3)           /* a CUDA call failed */
#define MOCHY_E_TIMEOUT (-4)        /* a bounded device wait ran out */
#define MOCHY_E_NOT_PROJECTED (-5)  /* the call needs mochy_project first */
#define MOCHY_E_UNSUPPORTED (-6)    /* outside the limits above */
#define MOCHY_E_BUSY (-7)           /* serving queue full */
#define MOCHY_W_DEGENERATE_CP 1     /* success, but every significance is 0 */

#define MOCHY_N_H 26
#define MOCHY_N_3H 431
#define MOCHY_MAX_EDGE_SIZE 63
#define MOCHY_MAX_EDGES ((1 << 26) - 1)

#define MOCHY_A 1       /* MoCHy-A: hyperedge sampling (Algorithm "sampling_ver1") */
#define MOCHY_A_PLUS 2  /* MoCHy-A+: hyperwedge sampling (Algorithm "sampling_ver2") */

typedef struct mochy_ctx mochy_ctx;

typedef struct {
  int32_t theta;            /* 3h-motif threshold theta >= 1 (Section 4.1); 1 */
  double eps;               /* epsilon of Eq. "significance"; 1.0 */
  int64_t hbm_budget_bytes; /* device bytes the context may hold; 0 = no cap */
  int32_t device;           /* CUDA device ordinal; 0 */
  void* stream;             /* cudaStream_t to run on; NULL = own stream */
  int32_t exact_kernel;     /* mochy_count_exact: 0 = split (open pairs counted
                               per centre, closed ones enumerated), 1 = plain
                               per-hyperwedge scan; both give the same counts */
  int32_t dense_threshold;  /* split kernel: line degree from which a row is
                               kept as a bitmap; 0 = chosen by the tuner */
  int32_t rest_path;        /* split kernel, closed candidates of dense rows
                               outside the popcounted combinations: 1 = each
                               lane classifies those of its own word, 2 = they
                               are spread over the warp 32 at a time, 0 = 1 when
                               the dense rows span at least 2,048 words of 32
                               rows, else 2 (a batch always spreads them); all
                               give the same counts */
} mochy_config;

/* Fill *cfg with the defaults above. */
void mochy_config_default(mochy_config* cfg);

/* Create a context on cfg->device (cfg may be NULL for defaults).  Builds the
 * motif lookup tables on the device.  *out receives the handle. */
int mochy_create(mochy_ctx** out, const mochy_config* cfg);

/* Free the context and all its device memory.  NULL is accepted. */
int mochy_destroy(mochy_ctx* ctx);

/* Load a hypergraph G = (V, E) (Section 2.1).  Hyperedge i lists nodes
 * h_edge_nodes[h_edge_offsets[i] .. h_edge_offsets[i+1]) (host int64 offsets,
 * n_edges + 1 of them, starting at 0; int32 node ids in [0, n_nodes)).  A
 * hyperedge must be non-empty and list each node once, in any order.  E is a
 * set (Section 2.1 footnote): repeated hyperedges are dropped, the first
 * occurrence is kept, and hyperedge ids are positions after that removal.
 * Any previous hypergraph and line graph of ctx are released.
 * *n_duplicates_removed (may be NULL) receives the number dropped.
 * Errors: MOCHY_E_INVALID for malformed input, MOCHY_E_UNSUPPORTED past the
 * limits. */
int mochy_load(mochy_ctx* ctx, int64_t n_nodes, int64_t n_edges,
               const int64_t* h_edge_offsets, const int32_t* h_edge_nodes,
               int64_t* n_duplicates_removed);

/* As mochy_load, with the two arrays already in device memory (not kept). */
int mochy_load_device(mochy_ctx* ctx, int64_t n_nodes, int64_t n_edges,
                      const int64_t* d_edge_offsets, const int32_t* d_edge_nodes,
                      int64_t* n_duplicates_removed);

/* Number of hyperedges and node-list length of the loaded hypergraph; with
 * non-NULL host arrays (n_edges + 1 and n_incidences entries) also copies
 * the deduplicated CSR out (node lists sorted ascending). */
int mochy_get_hypergraph(mochy_ctx* ctx, int64_t* n_nodes, int64_t* n_edges,
                         int64_t* n_incidences, int64_t* h_edge_offsets,
                         int32_t* h_edge_nodes);

/* Build the line graph (Section 2.1 "Line Graph"; Algorithm
 * "hyperwedge_counting", Section 3.1): for every hyperedge e_i the sorted
 * list of adjacent e_j with omega = |e_i & e_j|.  Kept on the device.
 * *n_wedges = |wedges| (hyperwedges), *max_line_degree = max |N_{e_i}|
 * (either may be NULL).  Needs enough device memory for 16 bytes per
 * hyperwedge. */
int mochy_project(mochy_ctx* ctx, int64_t* n_wedges, int32_t* max_line_degree);

/* Copy |N_{e_i}| for every hyperedge to h_degrees (n_edges int64). */
int mochy_line_degrees(mochy_ctx* ctx, int64_t* h_degrees);

/* Exact counts (MoCHy-E, Algorithm "exact_motif_counting", Section 3.2):
 * out_h[t-1] = number of instances of h-motif t, out_3h[t-1] of 3h-motif t
 * (Section 4.1, threshold cfg.theta).  Needs mochy_project. */
int mochy_count_exact(mochy_ctx* ctx, int64_t out_h[MOCHY_N_H],
                      int64_t out_3h[MOCHY_N_3H]);

/* The part of the exact count that Algorithm "exact_motif_counting" adds in
 * the outer-loop iterations of the hyperedges h_anchors[0..n_anchors)
 * (host int32 ids; an id may not repeat): open instances centred at an
 * anchor plus closed instances whose smallest id is an anchor.  Summed over
 * all hyperedges it equals mochy_count_exact. */
int mochy_count_exact_subset(mochy_ctx* ctx, const int32_t* h_anchors,
                             int64_t n_anchors, int64_t out_h[MOCHY_N_H],
                             int64_t out_3h[MOCHY_N_3H]);

/* The share of the rows h_rows[0..n_rows) (host int32 hyperedge ids; an id
 * may not repeat) in the split kernel's exact count (exact_kernel = 0).  The
 * split kernel counts open instances per centre from all pairs of its
 * neighbours: for a centre e_c and neighbours e_p, e_q whose overlaps with
 * e_c fit in it, the pair is classified "as if open" (the regions of Lemma
 * "motif:time" with omega(p, q) = 0 and no triple intersection); a closed
 * instance is then added at its first member in the kernel's row order,
 * with its as-if-open terms at its three centres taken off.  A row's share
 * is its pairs as if open plus those corrections of the closed instances it
 * owns, so shares can be negative; summed over all rows they give the exact
 * count of Algorithm "exact_motif_counting" (Section 3.2), since any fixed
 * order owns every closed instance once.  The row order puts rows of line
 * degree below the dense threshold T first, ascending by id, then the rows
 * of line degree >= T ascending by (line degree, id); T is
 * cfg.dense_threshold when set, else the tuner's choice (mochy_trace_read
 * reports it).  Meant for checking the kernel at full size on a sample of
 * rows.  Needs mochy_project; MOCHY_E_INVALID for the scan kernel or a
 * batch. */
int mochy_count_exact_rows(mochy_ctx* ctx, const int32_t* h_rows, int64_t n_rows,
                           int64_t out_h[MOCHY_N_H], int64_t out_3h[MOCHY_N_3H]);

/* Measured choice of the split kernel's dense threshold (the line degree
 * from which a row's overlaps are kept as bit-planes): for each of the
 * n_candidates thresholds (host int32, each >= 2; with n_candidates = 0 the
 * tuner's model choice m and m/4, m/2, 2m, 4m) the split structures are
 * built and the split count of one seeded sample of rows (each row kept
 * with probability sample_fraction by a SplitMix64 hash of (seed, row)) is
 * timed with CUDA events on the context's stream.  The fastest threshold
 * becomes the context's dense threshold for the following counts and is
 * written to *best (may be NULL); tried and ms (may be NULL; n_candidates
 * entries, 5 for the default list) receive each candidate and its time in
 * milliseconds, -1 where its structures did not fit (device memory or the
 * kernels' limits).  The
 * paper has no counterpart (its exact count has no such threshold).  Needs
 * mochy_project; MOCHY_E_INVALID for the scan kernel or a batch. */
int mochy_tune_dense_threshold(mochy_ctx* ctx, const int32_t* candidates, int32_t n_candidates,
                               double sample_fraction, uint64_t seed, int32_t* best,
                               int32_t* tried, double* ms);

/* Hyperedge profiles (Section 3.1, "Hyperedge Profile (HP)"; Section 4.1
 * for their 3h-motif form): hp_h[e * 26 + t - 1] is the number of instances
 * of h-motif t that include hyperedge e, hp_3h[e * 431 + t - 1] the same for
 * 3h-motif t (host arrays of n_edges rows; either may be NULL).  Instances
 * are enumerated one by one (the per-hyperwedge scan of MoCHy-E, each
 * attributed to its three hyperedges), so the call suits hypergraphs of up
 * to about 1e10 connected triples and at most 786,432 hyperedges; it needs
 * mochy_project and 3.5 KB of device memory per hyperedge while it runs.
 * Summed over hyperedges, the profiles are three times the motif counts. */
int mochy_hyperedge_profile(mochy_ctx* ctx, int64_t* hp_h, int64_t* hp_3h);

/* Star node profiles (Section 3.1, "Node Profile (NP)" with the star
 * ego-network of v: the hyperedges that contain v, kept whole):
 * np_h[v * 26 + t - 1] / np_3h[v * 431 + t - 1] count the instances of
 * h-motif / 3h-motif t among those hyperedges (host arrays of n_nodes rows;
 * either may be NULL).  Every such instance is a closed instance of G whose
 * triple intersection holds v, so a row sums to C(|E_v|, 3).  Instances are
 * enumerated one by one, as for mochy_hyperedge_profile (same size limits);
 * needs mochy_project and 3.5 KB of device memory per node while it runs.
 * Radial and contracted node profiles are not provided. */
int mochy_star_node_profile(mochy_ctx* ctx, int64_t* np_h, int64_t* np_3h);

/* Radial node profiles (Section 3.1, "Node Profile (NP)" with the radial
 * ego-network of v: node set V_v = the union of the hyperedges that contain
 * v, hyperedges R_v = the hyperedges that are subsets of V_v):
 * np_h[v * 26 + t - 1] / np_3h[v * 431 + t - 1] count the instances of
 * h-motif / 3h-motif t among the hyperedges of R_v (host arrays of n_nodes
 * rows; either may be NULL).  Hyperedges are kept whole, so every instance
 * is classified as in G.  One CTA per node marks V_v and R_v in bitmaps and
 * counts the instances among R_v (Algorithm "exact_motif_counting" with the
 * neighbours outside R_v skipped); the work is the sum over nodes of
 * sum_{e in R_v} |N_e|^2, so the call suits small hypergraphs.  Needs
 * mochy_project, 3.5 KB of device memory per node and (n_nodes / 8 +
 * n_edges * 4.2) bytes per resident CTA while it runs.  Rows of star
 * profiles (mochy_star_node_profile) never exceed these. */
int mochy_radial_node_profile(mochy_ctx* ctx, int64_t* np_h, int64_t* np_3h);

/* kh-motif counts (Section 4.1, "Extensions Beyond Ternary"): each of the
 * seven regions takes one of k states (2 <= k <= 4): 0 when empty, else 1
 * plus the number of the k - 2 ascending thresholds (host int32, values in
 * [1, 63]) its cardinality exceeds; k = 3 with threshold theta gives the
 * 3h-motifs, k = 4 has X(4) = 3,076 motifs (Appendix "Number of kH-motifs").
 * Patterns are canonicalised and filtered as for 3h-motifs and numbered in
 * ascending (parent h-motif id, canonical tuple) order (mochy_kh_pattern).
 * out_kh[t-1] (cap >= X(k) entries, may be NULL) receives the count of
 * kh-motif t, out_h (26, may be NULL) the h-motif counts, *n_motifs (may be
 * NULL) X(k).  Instances are enumerated one by one by the per-hyperwedge
 * scan (exact_kernel = 1's kernel, at most about 300,000 hyperedges).
 * Needs mochy_project. */
int mochy_count_kh(mochy_ctx* ctx, int32_t k, const int32_t* thresholds, int64_t* out_h,
                   int64_t* out_kh, int64_t cap, int64_t* n_motifs);

/* Region states (regions (1)..(7) of Section 2.2) of kh-motif `id` for k
 * states; MOCHY_E_INVALID for an id outside 1..X(k). */
int mochy_kh_pattern(mochy_ctx* ctx, int32_t k, int32_t id, uint8_t regions_out[7]);

/* Instance enumeration (MoCHy-E_ENUM, Algorithm "alg:enum", Section 3.2):
 * every instance of every motif, written once as a row of five int32
 * (i, j, k, h-motif id, 3h-motif id) with i < j < k hyperedge ids, into
 * h_out (host, capacity rows), in no particular order.  *n_instances
 * receives the number of instances (the sum of mochy_count_exact's counts);
 * when it exceeds capacity only `capacity` of them are written.  The rows
 * are produced on the device by the per-hyperwedge scan into a stream of
 * capacity * 20 bytes (budget-checked) and copied out.  Needs
 * mochy_project. */
int mochy_enumerate(mochy_ctx* ctx, int64_t capacity, int32_t* h_out, int64_t* n_instances);

/* Sampled counts.  method MOCHY_A draws `samples` hyperedges uniformly with
 * replacement (Algorithm "sampling_ver1"); MOCHY_A_PLUS draws `samples`
 * hyperwedges (Algorithm "sampling_ver2").  Draw n uses Philox4x32-10 with
 * counter (n_lo, n_hi, stream, 0), key (seed_lo, seed_hi), stream 1 for A and
 * 2 for A+, and maps the 64-bit output u to floor(u * range / 2^64);
 * hyperwedges are indexed in ascending (i, j), i < j.  raw_* receive the
 * int64 per-motif increments, est_* the unbiased estimates
 * raw * |E| / (3 samples) (A) or raw * |wedges| / (w[t] samples) (A+, w = 2
 * for open and 3 for closed motifs, Eq. "wt").  Output pointers may be NULL. */
int mochy_count_sampled(mochy_ctx* ctx, int method, int64_t samples, uint64_t seed,
                        int64_t raw_h[MOCHY_N_H], int64_t raw_3h[MOCHY_N_3H],
                        double est_h[MOCHY_N_H], double est_3h[MOCHY_N_3H]);

/* MoCHy-A+ without the line graph (Section 3.4, "Motif Counting without
 * Line Graphs"; Algorithms "alg_memdeg" and "alg_memdeg_adv"): the same
 * estimator as mochy_count_sampled(MOCHY_A_PLUS) with the same draws
 * (draw n is hyperwedge floor(u |wedges| / 2^64) of the ascending (i, j)
 * order, Philox4x32-10 counter (n_lo, n_hi, 2, 0), key seed), so raw counts
 * and estimates are identical to the projected call's, but it needs only
 * mochy_load: no line graph is built.  Neighbourhoods are never stored;
 * the hyperedge-id space is scanned per drawn hyperwedge with membership
 * bitmaps of the most popular nodes (as many as budget_bytes allows; <= 0:
 * a quarter of the context's budget, else 4 GiB) and the incidence lists of
 * the others.  The bitmaps, the line-graph degrees and their prefix are
 * built by the first call after a load and kept until the next load (the
 * budget of later calls is then ignored; results never depend on it).
 * *n_wedges (may be NULL) receives |wedges|.  Output pointers may be NULL.
 * With mochy_trace level 2, mochy_trace_read reports candidates, scanned
 * words, list entries and node-list classifications of the call. */
int mochy_count_sampled_onthefly(mochy_ctx* ctx, int64_t samples, uint64_t seed,
                                 int64_t budget_bytes, int64_t raw_h[MOCHY_N_H],
                                 int64_t raw_3h[MOCHY_N_3H], double est_h[MOCHY_N_H],
                                 double est_3h[MOCHY_N_3H], int64_t* n_wedges);

/* Sampled counts as mochy_count_sampled, written to caller-provided DEVICE
 * arrays (d_raw_h[26], d_raw_3h[431] int64; d_est_h[26], d_est_3h[431] FP64),
 * without allocating any device memory.  The paper has no counterpart: this
 * is for callers that cannot allocate while they run, such as a process whose
 * device memory is handed out by another runtime or pool, or a serving loop
 * with a fixed memory reservation.  Its working memory is one fixed array
 * inside the library (about 1.6 MB, held by every GPU that loads the library
 * until the process exits), so MOCHY_A takes at most 65,536 samples per call
 * (more returns MOCHY_E_UNSUPPORTED); MOCHY_A_PLUS has no limit.  The first
 * call on a device looks the array up (cudaGetSymbolAddress) and should come
 * before any stream capture; the address is kept for the process, so the
 * call must not be used on a device after cudaDeviceReset.  All calls share the array: calls whose GPU work
 * overlaps race, so run them one after another on the context's stream.
 * MOCHY_A waits for its stream once (to size its work); the outputs are
 * ready when the context's stream (mochy_stream) has completed. */
int mochy_count_sampled_noalloc(mochy_ctx* ctx, int method, int64_t samples, uint64_t seed,
                                int64_t* d_raw_h, int64_t* d_raw_3h, double* d_est_h,
                                double* d_est_3h);

/* One randomized hypergraph of the paper's null model into a new context
 * *out (same config): Chung-Lu on the incidence graph (Algorithm
 * "randomized_hypergraph_alg", Appendix "Randomized Hypergraphs") followed by
 * the set transform (Algorithm "transform"), empty hyperedges dropped and
 * repeated hyperedges dropped keeping the first.  Draw d of copy c uses
 * Philox4x32-10 with counter (d_lo, d_hi, 3 or 4, c) and key (seed); node
 * and hyperedge endpoints are chosen with probability proportional to degree
 * through integer prefix sums.  The copy is not projected. */
int mochy_randomize(mochy_ctx* src, uint64_t seed, uint32_t copy, mochy_ctx** out);

/* Significance and characteristic profile (Eq. "significance", Eq. "cp",
 * Section 3.1) of the loaded hypergraph against n_random randomized copies
 * (copies 0..n_random-1 of mochy_randomize with this seed), all counted
 * exactly; M_rand is the mean over copies.  FP64.  counts_h / counts_3h
 * (may be NULL) receive (1 + n_random) rows, the input first.  Returns
 * MOCHY_W_DEGENERATE_CP (and zero CPs) when all significances are 0. */
int mochy_profile(mochy_ctx* ctx, int32_t n_random, uint64_t seed,
                  double sig_h[MOCHY_N_H], double cp_h[MOCHY_N_H],
                  double sig_3h[MOCHY_N_3H], double cp_3h[MOCHY_N_3H],
                  int64_t* counts_h, int64_t* counts_3h);

/* Timings and sizes of a batched profile (mochy_profile_batch); times are
 * device milliseconds summed over waves. */
typedef struct {
  double ms_generate;   /* inputs loaded, copies drawn, transformed and loaded */
  double ms_project;    /* line graph of the union */
  double ms_prepare;    /* split structures (dense index, bitmaps) */
  double ms_count;      /* the one CUDA-graph launch of the counting kernels */
  double ms_finish;     /* per-hypergraph counts, significance, CP, copy-out */
  int64_t n_waves;      /* unions counted (1 unless memory forced a split) */
  int64_t n_units;      /* hypergraphs counted: n_graphs * (1 + n_random) */
  int64_t max_units_per_wave;
  int64_t n_edges;      /* hyperedges of the unions (after duplicate removal) */
  int64_t n_wedges;     /* hyperwedges of the unions */
  int64_t instances;    /* connected triples counted, all hypergraphs */
  int32_t dense_threshold;
} mochy_batch_info;

/* Significance and characteristic profiles (Eq. "significance", Eq. "cp",
 * Section 3.1) of n_graphs hypergraphs at once: for graph g, exactly what
 * mochy_profile computes for it with n_random copies and seed seeds[g].
 * Graph g has n_nodes[g] >= 1 nodes and n_edges[g] hyperedges given as
 * edge_offsets[g] (n_edges[g] + 1 entries from 0) and edge_nodes[g] (host
 * arrays, copied; repeated hyperedges are dropped keeping the first).  The
 * inputs and their randomized copies are generated on the device, as one
 * disjoint union per wave (as many inputs as the configured memory budget,
 * else 70% of the free device memory, allows), and every hypergraph of the
 * union is counted exactly by one launch of a CUDA graph of persistent
 * work-queue kernels.  Outputs (host, caller-allocated, each may be NULL):
 * sig_h, cp_h [n_graphs][26]; sig_3h, cp_3h [n_graphs][431]; counts_h
 * [n_graphs][1 + n_random][26] and counts_3h [n_graphs][1 + n_random][431]
 * (the input first, then copies 0..); degenerate [n_graphs] (1 when all
 * significances of h- or 3h-motifs are 0); info.  cfg gives theta, eps,
 * device, budget and dense threshold (its stream is ignored: the batch runs
 * on streams of its own; exact_kernel must be 0).  The environment variable
 * MOCHY_BATCH_MAX_GRAPHS, when set to a positive number, caps the inputs per
 * wave.  Returns MOCHY_W_DEGENERATE_CP when any graph is degenerate. */
int mochy_profile_batch(const mochy_config* cfg, int32_t n_graphs, const int64_t* n_nodes,
                        const int64_t* n_edges, const int64_t* const* edge_offsets,
                        const int32_t* const* edge_nodes, int32_t n_random,
                        const uint64_t* seeds, double* sig_h, double* cp_h, double* sig_3h,
                        double* cp_3h, int64_t* counts_h, int64_t* counts_3h,
                        int32_t* degenerate, mochy_batch_info* info);

/* ---- Serving ------------------------------------------------------------
 * A server answers a stream of requests on one GPU with continuous
 * batching: n_slots worker threads, each with a context and a CUDA stream of
 * its own, take queued requests in arrival order as soon as a slot is free
 * and the request's estimated device memory fits the budget beside the
 * requests already running (a later request that fits may start before an
 * earlier one that does not, but at most 32 times for any one request:
 * then later requests wait until it fits) (cfg->hbm_budget_bytes, else 70% of the device
 * memory free at creation), so requests that arrive while others run start
 * as slots and memory free up and their work overlaps on the device.  A
 * request runs exactly the calls a direct caller would make (mochy_load,
 * mochy_project, then mochy_count_exact, mochy_count_sampled or
 * mochy_profile) on a context of its own: its result is the same alone and
 * in any mix.  A MoCHy-A+ request whose line graph would take more than a
 * quarter of the budget runs without one (mochy_count_sampled_onthefly,
 * identical results, n_wedges reported the same way), so hypergraphs whose
 * line graph does not fit the device can still be served.  The functions
 * may be called from any host thread. */
typedef struct mochy_server mochy_server;

#define MOCHY_REQ_EXACT 1    /* exact counts (Algorithm "exact_motif_counting") */
#define MOCHY_REQ_SAMPLED 2  /* sampled counts (method, samples, seed) */
#define MOCHY_REQ_PROFILE 3  /* significance and CP (n_random, seed) */

typedef struct {
  int32_t kind;                 /* MOCHY_REQ_* */
  int64_t n_nodes, n_edges;     /* the hypergraph, as for mochy_load (host */
  const int64_t* edge_offsets;  /* arrays, copied at submission) */
  const int32_t* edge_nodes;
  int32_t method;               /* sampled: MOCHY_A or MOCHY_A_PLUS */
  int64_t samples;              /* sampled: number of draws */
  int32_t n_random;             /* profile: randomized copies */
  uint64_t seed;                /* sampled and profile */
} mochy_request;

typedef struct {
  int32_t status;                   /* MOCHY_OK, MOCHY_W_DEGENERATE_CP or an error */
  int64_t n_wedges;                 /* hyperwedges of the request's hypergraph */
  int64_t counts_h[MOCHY_N_H];      /* exact counts; sampled raw counts; profile: */
  int64_t counts_3h[MOCHY_N_3H];    /*   counts of the input */
  double est_h[MOCHY_N_H];          /* sampled: estimates */
  double est_3h[MOCHY_N_3H];
  double sig_h[MOCHY_N_H], cp_h[MOCHY_N_H];      /* profile */
  double sig_3h[MOCHY_N_3H], cp_3h[MOCHY_N_3H];
  double queue_ms, service_ms, latency_ms;       /* host clock, submission to result */
  char error[128];                  /* message of a failed request, else empty */
} mochy_result;

typedef struct {
  int64_t submitted, completed, failed, rejected, queued, in_flight, peak_in_flight;
  int64_t budget_bytes, peak_reserved_bytes;
  double p50_ms, p99_ms, mean_ms, max_ms;   /* latency of completed requests (nearest rank) */
  double throughput_rps;                    /* completed / (last completion - first submission) */
} mochy_serving_stats;

/* Start a server with n_slots (1..64) workers and room for max_queue queued
 * requests. */
int mochy_server_create(mochy_server** out, const mochy_config* cfg, int32_t n_slots,
                        int32_t max_queue);

/* Queue a request; *ticket identifies it.  MOCHY_E_NOMEM when its estimated
 * memory exceeds the whole budget, MOCHY_E_BUSY when the queue is full,
 * MOCHY_E_INVALID for a malformed request. */
int mochy_server_submit(mochy_server* s, const mochy_request* req, int64_t* ticket);

/* Result of a ticket: returns 1 and fills *out (once; the ticket is then
 * forgotten) when done, 0 when not done within wait_ms milliseconds. */
int mochy_server_poll(mochy_server* s, int64_t ticket, mochy_result* out, int32_t wait_ms);

/* Counters and latency percentiles so far. */
int mochy_server_stats(mochy_server* s, mochy_serving_stats* st);

/* Stop the workers after the requests they are running; queued requests are
 * dropped.  NULL is accepted. */
int mochy_server_destroy(mochy_server* s);

/* Region pattern of motif `id` (kind 2: h-motif, kind 3: 3h-motif): states
 * of regions (1)..(7) of Section 2.2 (0 empty, 1 at most theta nodes, 2 more;
 * h-motifs use 0/1). */
int mochy_motif_pattern(int kind, int32_t id, uint8_t regions_out[7]);

/* cudaStream_t the context runs on (as void*), for event timing. */
void* mochy_stream(mochy_ctx* ctx);

/* Tracing of the exact count: level 1 records the duration of each of its
 * phases (CUDA events on the context's stream, no effect on the kernels);
 * level 2 also counts kernel statistics (scanned words, candidates, cycles
 * per section), which slows the kernels; 0 turns tracing off.
 * mochy_trace_read writes the last traced call as one JSON object into buf
 * (len bytes).  The environment variable MOCHY_TRACE=1 selects level 2 for
 * every context and also prints to stderr. */
int mochy_trace(mochy_ctx* ctx, int level);
int mochy_trace_read(mochy_ctx* ctx, char* buf, int64_t len);

/* Bytes of device memory the context holds now. */
int64_t mochy_device_bytes(mochy_ctx* ctx);

/* Number of kernels the library launched in this process (for accounting). */
int64_t mochy_kernel_launches(void);

const char* mochy_strerror(int code);
const char* mochy_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MOCHY_H */
