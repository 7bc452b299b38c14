/*
 * tn.h -- C-ABI of the GB300 contraction-tree executor (libtn.so).
 *
 * Executes a given contraction tree, optionally sliced, over a tensor
 * network of real or complex tensors on one GPU (sm_103a).  The problem is
 * the one stated in Sec. 2 of arXiv 2002.01935 (Gray & Kourtis,
 * "Hyper-optimized tensor network contraction"): a network is a graph whose
 * vertices carry tensors T_v over ordered index tuples t_v and whose edges
 * carry discrete labels of size w(e); a rooted binary contraction tree
 * fixes the order of pairwise contractions; slicing (Sec. 4.7.1) moves the
 * sums over a chosen set of labels outside and sums the independent sliced
 * contractions.
 *
 * Conventions shared by every call:
 *   - Labels are arbitrary int64 ids.  A label may occur in any number of
 *     tensors: in two it is an ordinary edge, in more a hyperedge (Sec. 3.5);
 *     in one and not open it is summed when that tensor is first contracted.
 *     A label repeated inside one tensor is rejected (no self loops, Sec. 2).
 *   - Tensors are dense and row-major over their label order (the last label
 *     varies fastest).  TN_C64 stores interleaved (re, im) float32 pairs,
 *     TN_R32 plain float32.
 *   - Results are returned in FP64 as (mantissa, exponent): value =
 *     mantissa * 2^exp2.  Every contraction is renormalised by a power of
 *     two (Sec. 4.2, "actively renormalizing"), so values far outside the
 *     float range are representable.
 *   - No call throws.  A non-OK status leaves outputs untouched; the message
 *     of the last failure on the calling thread is returned by
 *     tn_last_error().
 *   - All device work is ordered on the caller's CUDA stream (a
 *     cudaStream_t passed as void*; NULL = legacy default stream).
 *   - Power-of-two label sizes run on the tiled kernels; other sizes run on
 *     the generic kernel (same results, slower).
 */
#ifndef TN_H
#define TN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tn_net tn_net; /* opaque, library-owned */

typedef enum {
    TN_OK = 0,
    TN_EINVAL = 1,        /* malformed network, tree, labels or arguments   */
    TN_ENOMEM = 2,        /* device or host allocation failed               */
    TN_ECUDA = 3,         /* a CUDA runtime call failed                     */
    TN_ETIMEOUT = 4,      /* a bounded device-side wait gave up             */
    TN_EUNSUPPORTED = 5   /* valid request the executor cannot run          */
} tn_status;

typedef enum {
    TN_R32 = 0,           /* real float32 leaves                            */
    TN_C64 = 1            /* complex64 leaves, interleaved (re, im)         */
} tn_dtype;

/*
 * Arithmetic used inside each pairwise contraction (the cross-slice sum is
 * always FP64).  Complex products are formed from four real products (4M)
 * or, where named, three (3M: Re A Re B, Im A Im B and (Re A + Im A)(Re B +
 * Im B)).
 *   TN_MODE_FP32       : FP32 FMA on CUDA cores (plain complex64 / float32)
 *   TN_MODE_TF32_3M    : operands rounded to TF32, one tensor-core pass,
 *                        3M for complex nodes with >= 128 columns on both
 *                        sides (4M otherwise), FP32 accumulation
 *   TN_MODE_TF32_SPLIT : operands split hi+lo in TF32, three products
 *                        (hi*hi + hi*lo + lo*hi), 4M, FP32 accumulation
 *   TN_MODE_BF16_SPLIT : the same split in BF16
 *   TN_MODE_FP16_SPLIT : the same split in FP16, whose 11-bit significand
 *                        equals TF32's while its tensor-core rate equals
 *                        BF16's.  Each operand is scaled by a power of two
 *                        so that its largest magnitude lies in [2^14, 2^15);
 *                        entries at least 2^-18 of that largest keep the full
 *                        22 bits of hi + lo, smaller ones lose low bits (FP16
 *                        subnormals) and those below 2^-40 of it count as 0.
 *                        Suited to networks whose tensors span a moderate
 *                        dynamic range (random circuits); prefer TF32_SPLIT
 *                        where single tensors span more than ~2^18.
 * Nodes too small for the tensor cores run the FP32 path in every mode.
 */
typedef enum {
    TN_MODE_FP32 = 0,
    TN_MODE_TF32_3M = 1,
    TN_MODE_TF32_SPLIT = 2,
    TN_MODE_BF16_SPLIT = 3,
    TN_MODE_FP16_SPLIT = 4
} tn_mode;

enum { TN_MEM_DEVICE = 0, TN_MEM_HOST = 1 };

/*
 * tn_create -- build a network handle from tensor shapes and labels
 * (Sec. 2: the graph G, the tuples t_v and the weights w(e) = |D(e)|).
 *   dt           storage type of every leaf.
 *   n_tensors    |V| >= 1.
 *   ranks[v]     number of labels of tensor v (0 allowed: a scalar).
 *   labels       the concatenated t_v tuples, sum(ranks) int64 ids.
 *   n_labels, label_ids[i], label_dims[i]
 *                every label used, with its size w(e) >= 1.
 *   n_open, open_labels
 *                labels left uncontracted, in the order of the output
 *                tensor's axes (row-major).  n_open = 0: a scalar network.
 * The arrays are copied; the caller keeps ownership.  On success *out owns a
 * handle to be released with tn_destroy.  Errors: TN_EINVAL (unknown or
 * duplicate label, repeated label in a tensor, open label not in any tensor,
 * size < 1), TN_EUNSUPPORTED (a tensor of more than 2^40 entries), TN_ENOMEM.
 */
tn_status tn_create(tn_net **out, tn_dtype dt, int32_t n_tensors, const int32_t *ranks,
                    const int64_t *labels, int32_t n_labels, const int64_t *label_ids,
                    const int64_t *label_dims, int32_t n_open, const int64_t *open_labels);

/*
 * tn_set_tensor -- attach the entries of leaf v (T_v of Sec. 2).
 *   ptr   row-major entries in the label order given to tn_create.
 *   mem   TN_MEM_DEVICE: a device pointer, borrowed (not copied): it must
 *         stay valid and unchanged until every contraction that reads it
 *         has completed on its stream.
 *         TN_MEM_HOST: a host pointer, read by every later tn_contract:
 *         during the call all host leaves are gathered into one library-
 *         owned page-locked image, which goes to the device as one copy on
 *         the call's stream (under stream capture: one copy per leaf, read
 *         when the graph runs).
 * Errors: TN_EINVAL (v out of range, ptr NULL for a non-empty tensor).
 */
tn_status tn_set_tensor(tn_net *net, int32_t v, const void *ptr, int32_t mem);

/*
 * Per-call options of tn_contract_ex.  Zero-initialise, then set fields.
 *   slice_begin, slice_count
 *       contract only slices [slice_begin, slice_begin + slice_count) of the
 *       d_sliced = prod w(e) slices (slice_count <= 0: all).  Slice id s
 *       fixes the sliced labels to the mixed-radix digits of s, the last
 *       listed label varying fastest (Sec. 4.7.1).
 *   no_graph
 *       1: launch the per-slice node sequence directly instead of replaying
 *       a captured CUDA graph.
 *   reserved0
 *       must be 0 (kernel choices come from the plan, see tn_autotune).
 *   prof_events, prof_first, prof_count
 *       timing hooks: prof_events[i] is recorded on the stream just before
 *       launch step prof_first+i of the per-slice sequence (steps as listed
 *       by tn_plan_steps) and prof_events[prof_count] just after step
 *       prof_first+prof_count-1, in every slice (the last slice's records
 *       win).  The events are caller-owned timing events.
 *   slice_batch
 *       slice-parallel execution: every node launch runs this many
 *       consecutive slices side by side (each with its own workspace copy,
 *       so memory grows by this factor); their results are folded into the
 *       FP64 sum in slice order, so the result does not depend on it.
 *       0 or 1: one slice per launch.
 *   persistent
 *       1: the whole call in one persistent dataflow launch (Sec. 4.7.1:
 *       the slices are independent): every node of every slice of the call
 *       side by side -- small or narrow nodes as chunks of outputs, nodes
 *       with >= 32 rows and columns and >= 4096 outputs as 64 x 64 output
 *       tiles over all of K -- taken in tree order by resident CTAs that
 *       wait (bounded) for their inputs' completion counters; then one fold
 *       of the slices' roots, in slice order, into the FP64 result on the
 *       device.  Every node runs in FP32 on the CUDA cores (the mode's tensor
 *       cores are not used); slice_batch is ignored (all slices of the call
 *       run side by side, as many as 8 GiB of workspace copies hold; more
 *       slices take several such launches).  Needs power-of-two label sizes
 *       (else TN_EUNSUPPORTED).  0: the per-step launch sequence.
 */
typedef struct {
    int64_t slice_begin;
    int64_t slice_count;
    int32_t no_graph;
    int32_t reserved0;
    void *const *prof_events; /* NULL, or prof_count+1 cudaEvent_t (as void*) */
    int32_t prof_first;
    int32_t prof_count;
    int32_t slice_batch;      /* slices run side by side per launch (>= 1) */
    int32_t persistent;       /* 1: one persistent launch for the whole call */
    int32_t reserved[4];
} tn_options;

/*
 * tn_contract -- contract the network with the given tree and slicing.
 *   tree_pairs   2*(n_tensors-1) int32 ids: internal vertex n_tensors+i has
 *                children (tree_pairs[2i], tree_pairs[2i+1]); leaves are
 *                0..n_tensors-1, every id is used exactly once and a child id
 *                is smaller than its parent's; the root is last (the l(v),
 *                r(v) tuples of Sec. 2).  A node keeps a label iff it is
 *                open or occurs in a leaf outside the node's subtree
 *                (Eq. incidence, generalised to hyperedges and open labels).
 *   n_sliced, sliced_labels
 *                labels summed outside the tree (Sec. 4.7.1); they must be
 *                non-open labels of the network.
 *   mode         arithmetic of the node contractions (tn_mode).
 *   out          FP64 mantissa of the result over the open labels in
 *                tn_create order: complex128 (TN_C64) or float64 (TN_R32),
 *                prod(open sizes) entries (1 for a scalar network).
 *   out_mem      TN_MEM_DEVICE or TN_MEM_HOST, for out and out_exp2.
 *   out_exp2     one int64: value = out * 2^(*out_exp2).
 *   stream       cudaStream_t (as void*).
 * Device outputs are written asynchronously on the stream; host outputs
 * are complete when the call returns (the call synchronises the stream).
 * The first call with a new (tree, slicing, mode) plans the nodes and
 * allocates the workspace (cached in the handle; a call during stream
 * capture must reuse a cached plan).  Errors: TN_EINVAL (malformed tree,
 * sliced label open or unknown, a leaf without data), TN_EUNSUPPORTED (an
 * intermediate of the sliced tree with more than 2^40 entries, or a node of
 * more than 2^62 multiply-adds), TN_ENOMEM, TN_ECUDA, TN_ETIMEOUT.
 */
tn_status tn_contract(tn_net *net, const int32_t *tree_pairs, int32_t n_sliced,
                      const int64_t *sliced_labels, tn_mode mode, void *out, int32_t out_mem,
                      int64_t *out_exp2, void *stream);

/* tn_contract with options (NULL options = tn_contract). */
tn_status tn_contract_ex(tn_net *net, const int32_t *tree_pairs, int32_t n_sliced,
                         const int64_t *sliced_labels, tn_mode mode, const tn_options *opt,
                         void *out, int32_t out_mem, int64_t *out_exp2, void *stream);

/*
 * tn_contract_grad -- reverse-mode derivative of the contraction with
 * respect to every leaf.  The paper states only the forward problem; the
 * backward pass is the adjoint of each pairwise contraction: for a node
 * C = A * B with adjoint Cbar, Abar = contract(Cbar, conj(B)) over B's
 * labels not in A, and Bbar likewise, applied root to leaves.  Forward
 * intermediates are recomputed per slice, not stored across slices.
 *   out_adjoint  host FP64 array shaped like tn_contract's out (complex128
 *                or float64), the adjoint of the result's mantissa:
 *                the result's adjoint is out_adjoint * 2^(adj_exp2).
 *   leaf_grads   n_tensors device pointers (NULL to skip a leaf), each
 *                shaped like the leaf (dtype dt): on return (in stream
 *                order) leaf_grads[v] = conj(d value / d T_v) * adjoint,
 *                summed over slices and contracted over the open labels --
 *                the convention of torch.autograd for complex tensors.
 *   Other arguments as tn_contract.  Errors as tn_contract.
 */
tn_status tn_contract_grad(tn_net *net, const int32_t *tree_pairs, int32_t n_sliced,
                           const int64_t *sliced_labels, tn_mode mode, const double *out_adjoint,
                           int64_t adj_exp2, void *const *leaf_grads, void *stream);

/* tn_contract_grad_ex flag: add the gradients into leaf_grads (which then
 * hold the caller's running sums) instead of overwriting them. */
#define TN_GRAD_ACCUMULATE 1u
/* tn_contract_grad_instances flag: the forward intermediates are those of the
 * last tn_contract_instances_keep call (same tree, mode, copies, strides and
 * leaf data): the sweep runs without recomputing them. */
#define TN_GRAD_KEPT_FORWARD 2u

/*
 * tn_contract_grad_ex -- tn_contract_grad with the adjoint in device memory
 * and/or accumulation into the gradient buffers, for loops over many
 * networks of one shape (e.g. the bitstrings of a circuit sharing a tree)
 * that sum their gradients without host round trips.
 *   out_adjoint   FP64 adjoint as in tn_contract_grad, in host memory
 *                 (adj_mem = TN_MEM_HOST: copied before the call returns)
 *                 or device memory (TN_MEM_DEVICE: read in stream order, so
 *                 it may come from earlier work on the stream, e.g. the
 *                 forward result, without a host synchronisation).
 *   adj_exp2      power-of-two exponent of the adjoint (host value).
 *   adj_exp2_dev  NULL, or (device adjoints only) a device int64 added to
 *                 adj_exp2 in stream order -- e.g. the negated exponent of
 *                 a tn_contract result, for adjoints such as 1 / value.
 *   flags         0 or TN_GRAD_ACCUMULATE.
 *   slice_begin, slice_count
 *                 the slices swept: [slice_begin, slice_begin + slice_count)
 *                 of the d_sliced slices (slice_count <= 0: all).  Partial
 *                 ranges give the gradient of that part of the sum: ranks
 *                 sharing the slices add their gradients (one all-reduce).
 *   Other arguments as tn_contract_grad.
 * Both calls keep, per (tree, slicing, mode), a library image of the leaves
 * (refreshed from the attached pointers at the start of every call) and of
 * the gradients, so that the per-slice launch sequence -- forward recompute,
 * reverse sweep, leaf gathers -- is one CUDA graph captured on the first
 * call and replayed by later calls whatever their pointers.  Neither call
 * may be made while the stream is being captured (TN_EUNSUPPORTED).  Calls
 * on one network must be ordered (one stream): they share that state.
 * Errors: as tn_contract; TN_EINVAL for a bad adj_mem, unknown flags, or
 * adj_exp2_dev with a host adjoint.
 */
tn_status tn_contract_grad_ex(tn_net *net, const int32_t *tree_pairs, int32_t n_sliced,
                              const int64_t *sliced_labels, tn_mode mode, const double *out_adjoint,
                              int32_t adj_mem, int64_t adj_exp2, const int64_t *adj_exp2_dev,
                              void *const *leaf_grads, uint32_t flags, int64_t slice_begin,
                              int64_t slice_count, void *stream);

/*
 * tn_contract_grad_instances -- the reverse sweep of n_inst copies of the
 * network in one launch sequence, the gradient counterpart of
 * tn_contract_instances (e.g. the bitstrings of one circuit: their networks
 * differ only in the output-state leaves).  Copy i reads leaf v at the
 * attached pointer plus i * leaf_inst_stride[v] elements (0, or NULL for
 * all: shared by every copy; otherwise at least the leaf's size).  Every
 * node launch covers all copies (each copy has its own workspace, packing
 * buffer and scale slots); slicing is allowed (every copy runs every
 * slice).
 *   out_adjoint   n_inst adjoints, each shaped like tn_contract's out (FP64,
 *                 complex (re, im) pairs), copy after copy; host or device
 *                 memory as adj_mem.
 *   adj_exp2      exponent added to every copy's adjoint.
 *   adj_exp2_dev  NULL, or (device adjoints only) n_inst device int64s,
 *                 copy i's adjoint exponent is adj_exp2 + adj_exp2_dev[i].
 *   leaf_grads    n_tensors device pointers (NULL: skipped): for a shared
 *                 leaf the sum over the copies of their gradients (added in
 *                 copy order); for a varying leaf copy i's gradient at
 *                 + i * leaf_inst_stride[v] elements.
 *   flags         TN_GRAD_ACCUMULATE and/or TN_GRAD_KEPT_FORWARD (below).
 *   slice_begin, slice_count  as tn_contract_grad_ex.
 * The device state grows to n_inst copies of the sweep's workspace; a
 * different (n_inst, shared/varying pattern) rebuilds it (and synchronises
 * the stream).  Errors: as tn_contract_grad_ex; TN_EINVAL for n_inst < 1
 * or overlapping copies; TN_EUNSUPPORTED when a node's launch grid would
 * exceed the CUDA limit for this many copies.
 */
tn_status tn_contract_grad_instances(tn_net *net, const int32_t *tree_pairs, int32_t n_sliced,
                                     const int64_t *sliced_labels, tn_mode mode, int32_t n_inst,
                                     const int64_t *leaf_inst_stride, const double *out_adjoint,
                                     int32_t adj_mem, int64_t adj_exp2, const int64_t *adj_exp2_dev,
                                     void *const *leaf_grads, uint32_t flags, int64_t slice_begin,
                                     int64_t slice_count, void *stream);

/*
 * tn_contract_instances_keep -- tn_contract_instances (unsliced scalar
 * networks, same arguments and outputs) computed in the state of the
 * reverse sweep of (tree, unsliced, mode) for n_inst copies, with every
 * intermediate kept.  A following tn_contract_grad_instances call with the
 * same tree, mode, n_inst and leaf strides, no slicing, and flag
 * TN_GRAD_KEPT_FORWARD then runs only the sweep: for an unsliced tree the
 * forward is computed once per gradient step instead of twice.  The library
 * refuses the flag (TN_EINVAL) when the kept state is gone (another
 * gradient call of that tree and mode ran in between, or another copy
 * count); it cannot see changes of the leaf data, which the caller must
 * not make in between.  Errors as tn_contract_instances; TN_EUNSUPPORTED
 * for sliced trees or open outputs.
 */
tn_status tn_contract_instances_keep(tn_net *net, const int32_t *tree_pairs, tn_mode mode, int32_t n_inst,
                                     const int64_t *leaf_inst_stride, double *out, int64_t *out_exp2,
                                     int32_t out_mem, void *stream);

/*
 * tn_contract_noalloc -- tn_contract for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a deployment variant.
 * tn_contract obtains its workspace with cudaMalloc on the first run of a
 * tree.  Hosts that must not allocate device memory after start-up (fixed
 * memory budgets, real-time loops) and processes whose device memory is
 * owned by another allocator's pool cannot let it do so.  This call runs the
 * same contraction on the generic node kernel (FP32 arithmetic, as
 * TN_MODE_FP32) with every piece of scratch -- intermediate tensors,
 * renormalisation slots, control block, FP64 accumulator -- inside one
 * fixed 8 MiB device array that is part of the library image; it calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *   Arguments as tn_contract (no mode); the leaves must be device pointers.
 *   Host outputs (out_mem = TN_MEM_HOST) make the call wait for the stream;
 *   on a stream that is capturing they are refused with TN_EUNSUPPORTED.
 *   Limit: the tree's workspace plus bookkeeping must fit in 8 MiB
 *   (tn_plan_info out[4] is the workspace part); larger trees are refused
 *   with TN_EUNSUPPORTED and a message giving the bytes needed.
 *   The first call on a device looks up the array's device address (with
 *   that device current); make that first call before any stream capture.
 *   Every GPU that loads the library holds the array until the process
 *   exits.  All calls share it and it keeps the last call's contents; each
 *   call clears what it needs cleared.  Calls whose GPU work overlaps (other
 *   streams, other threads) race on the array and must be serialised by the
 *   caller.
 */
tn_status tn_contract_noalloc(tn_net *net, const int32_t *tree_pairs, int32_t n_sliced,
                              const int64_t *sliced_labels, void *out, int32_t out_mem,
                              int64_t *out_exp2, void *stream);

/*
 * tn_contract_instances -- n_inst independent copies of one scalar network
 * (same labels and tree, unsliced) in one launch sequence: e.g. many output
 * bitstrings of one circuit (Eq. trans-amp), whose networks differ only in
 * their output tensors.  Copy i reads leaf v at the pointer attached with
 * tn_set_tensor plus i * leaf_inst_stride[v] elements (0: shared by all
 * copies; NULL: all shared); leaves must be device pointers.
 *   out        2 doubles per copy: FP64 mantissa (complex (re, im); real
 *              (x, 0)); out_exp2: one int64 per copy; out_mem as
 *              tn_contract.
 * Each copy count has its own plan, kept in the handle: its kernel choices
 * and K splits count the copies that share every launch (tn_autotune, which
 * times single copies, does not touch it), and its device state holds
 * n_inst workspace copies.  Errors: TN_EINVAL, TN_EUNSUPPORTED (open
 * labels, slicing, host leaves, stream capture), TN_ENOMEM, TN_ECUDA.
 */
tn_status tn_contract_instances(tn_net *net, const int32_t *tree_pairs, tn_mode mode, int32_t n_inst,
                                const int64_t *leaf_inst_stride, double *out, int64_t *out_exp2,
                                int32_t out_mem, void *stream);

/*
 * tn_plan_info -- cost figures of a (tree, slicing) for this network, from
 * Eqs. edgecon and vertexcon: out[0] = W_s (sliced width, log2 of the
 * largest tensor), out[1] = C (contraction cost of one slice), out[2] =
 * d_sliced, out[3] = FLOPs of all slices (8 C d_sliced complex, 2 C
 * d_sliced real), out[4] = workspace bytes per slice, out[5] = number of
 * nodes run by the tiled kernels, out[6] = by the tensor-core kernel,
 * out[7] = by the generic kernel.  Host only; no device work.
 */
tn_status tn_plan_info(tn_net *net, const int32_t *tree_pairs, int32_t n_sliced,
                       const int64_t *sliced_labels, tn_mode mode, double out[8]);

/*
 * tn_autotune -- per-node kernel choice by measurement.
 * For every tree node that runs alone in its launch step on a tiled or
 * tensor-core kernel, each candidate -- the five CUDA-core tile shapes
 * (64x64, 16x256, 4x1024, 256x16, 128x64 outputs per block, each with two
 * K splits) and, in the reduced-
 * precision modes, the tensor-core GEMM -- is launched once to warm up and
 * then reps times between two CUDA events on `stream`; the fastest is kept
 * in the handle's cached plan for (tree, sliced labels, mode) and used by
 * every later contraction with that plan (results agree within the mode's
 * tolerance whatever the choice).  Very large nodes that the tensor cores
 * can run skip the CUDA-core shapes.  The leaves must be attached; their
 * values do not matter.  choice (NULL or n_tensors-1 entries) receives per
 * node 0 (not tuned), 1..4 or 6 (tile shapes 64x64, 16x256, 4x1024,
 * 256x16, 128x64), 8 (tensor core), 9 (tensor core with 128-column
 * tiles where the planner's 256-column tiles fit: twice the CTAs, for
 * nodes with few tiles) or 10 (tensor core on the planar complex layout:
 * Re and Im planes of both operands, four real products per complex one
 * without interleaving or expanding either operand; complex nodes in a
 * split precision with at least 128 complex rows and columns).
 * Synchronises `stream`.  Errors as tn_contract.
 * Not in the paper: its executor has no kernel choices to tune.
 */
tn_status tn_autotune(tn_net *net, const int32_t *tree_pairs, int32_t n_sliced,
                      const int64_t *sliced_labels, tn_mode mode, int32_t reps, int32_t *choice,
                      void *stream);

/*
 * tn_selftest_flow_timeout -- failure-detection self-test of the bounded
 * device waits.  Launches one dataflow wave whose only item waits for a
 * completion counter that nothing raises; after its bound (about 2 s) the
 * wait gives up, the kernel records TN_ETIMEOUT in its control block and
 * returns, and the CUDA context stays usable.  Returns that status
 * (TN_ETIMEOUT; TN_OK would mean the wait did not run out) after
 * synchronising `stream`.  Uses 4 KB of device memory for the call.
 */
tn_status tn_selftest_flow_timeout(void *stream);

/*
 * tn_plan_steps -- the per-slice launch sequence of a plan (host only).
 * Nodes (0..n_tensors-2, tree order) run in launch steps: a wave step runs
 * all small nodes of one tree level in one launch, a single step runs one
 * node.  *n_steps receives the number of steps; if cap >= *n_steps, then
 * step_info[5*s..5*s+4] = (is_wave, kernel kind 0 generic / 1 tiled /
 * 2 tensor core, tile configuration, number of nodes, kernel launches of
 * the step) and step_nodes lists
 * the nodes of step 0, then step 1, ... (n_tensors-1 entries in all; may be
 * NULL).  Errors as tn_plan_info.
 */
tn_status tn_plan_steps(tn_net *net, const int32_t *tree_pairs, int32_t n_sliced,
                        const int64_t *sliced_labels, tn_mode mode, int32_t cap, int32_t *n_steps,
                        int32_t *step_info, int32_t *step_nodes);

/*
 * Batches of independent networks.  Sec. 4.7.1 of the paper notes that
 * independent contractions are embarrassingly parallel; a batch runs many
 * scalar networks (each with its own tree, no slicing) as one captured
 * launch sequence: per tree level, one launch covers the small nodes of
 * every network in the batch.
 *   tn_batch_create   n_nets handles and their trees (tree_pairs[i] as in
 *                     tn_contract for nets[i]); the handles must outlive the
 *                     batch and keep their leaves attached (device
 *                     pointers); allocates the merged device state.
 *   tn_batch_contract out: 2 doubles per network, the FP64 mantissa
 *                     (complex (re, im); real networks (x, 0));
 *                     out_exp2: one int64 per network (value = mantissa *
 *                     2^exp2); latency_ns (may be NULL): per network, the
 *                     time from the start of the batch until its root
 *                     contraction completed (%globaltimer, nanoseconds).
 *                     out_mem: TN_MEM_DEVICE or TN_MEM_HOST for all three.
 *   Errors: TN_EINVAL, TN_EUNSUPPORTED (open labels, slicing -- see
 *   tn_batch_create_sliced --, host leaves), TN_ENOMEM, TN_ECUDA.
 */
typedef struct tn_batch tn_batch;
tn_status tn_batch_create(tn_batch **out, int32_t n_nets, tn_net *const *nets,
                          const int32_t *const *tree_pairs, tn_mode mode);

/*
 * tn_batch_create_sliced -- tn_batch_create with a slicing per network
 * (Sec. 4.7.1): network i sums the n_sliced[i] labels sliced_labels[i]
 * outside its tree (n_sliced[i] = 0: unsliced).  Unsliced networks form the
 * merged forest as in tn_batch_create.  A sliced network stays out of it:
 * after the forest, on the same stream, its slices run through its own plan
 * -- up to 8 slices side by side per launch (fewer when their workspace
 * would exceed 2 GiB), folded in FP64 in slice order -- and its value,
 * exponent and latency (the time from the batch start until its last slice
 * was folded) go to the same outputs of tn_batch_contract.  Its device state
 * is that of its handle's plan (kept by the handle).  Errors as
 * tn_batch_create; TN_EINVAL for bad sliced labels (as tn_contract).
 */
tn_status tn_batch_create_sliced(tn_batch **out, int32_t n_nets, tn_net *const *nets,
                                 const int32_t *const *tree_pairs, const int32_t *n_sliced,
                                 const int64_t *const *sliced_labels, tn_mode mode);
tn_status tn_batch_contract(tn_batch *batch, double *out, int64_t *out_exp2, uint64_t *latency_ns,
                            int32_t out_mem, void *stream);
void tn_batch_destroy(tn_batch *batch);

/* Release the handle, its plans and its device memory (synchronises the
 * device work the handle issued).  NULL is ignored. */
void tn_destroy(tn_net *net);

/* Message of the last non-OK status on this thread ("" if none). */
const char *tn_last_error(void);

/* Library version string. */
const char *tn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TN_H */
