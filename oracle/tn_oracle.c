/*
 * tn_oracle.c -- plain CPU FP64 / complex128 contraction-tree executor.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark may load this library; the product path
 * never does.  It shares no code, header or table with the GPU executor.
 *
 * What it computes (arXiv 2002.01935):
 *   - The value of a tensor network is the |E| nested sums of the product of
 *     the entries of the |V| tensors (Sec. 4.7.1).  Open labels stay free.
 *   - A contraction tree only re-brackets that sum (Sec. 4.7.1); each tree
 *     vertex contracts its two children, taking the inner product over the
 *     shared labels (outer product if none), Sec. 2.
 *   - Node incidence (Sec. 2, Eq. incidence) generalised to hyperedges and
 *     open labels: a node keeps a label iff it is open or occurs in a leaf
 *     outside the node's subtree.
 *   - Slicing (Sec. 4.7.1): the sums over the sliced labels are moved
 *     outside; every fixed assignment gives a network with those labels
 *     removed, contracted with the same tree; the results are summed.
 *   - Active renormalisation (Sec. 4.2): after every contraction the node
 *     is scaled by 2^-e, e the frexp exponent of the largest |Re|,|Im|
 *     entry, and e is added to a running exponent, so values far outside
 *     the double range stay representable.
 *
 * Every node is evaluated by an explicit loop nest over the node's labels:
 * for each output entry, an odometer over the summed labels.  No BLAS, no
 * permutation tricks.  OpenMP splits the output entries across threads.
 *
 * Error codes: 0 ok, 1 invalid input, 2 out of memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>

typedef long long i64;

/* A dense tensor: labels in order, row-major, complex stored as (re, im). */
typedef struct {
    int rank;
    int *lab;       /* dense label indices */
    i64 size;
    double *re;
    double *im;     /* NULL for real networks */
    i64 exp2;       /* value = entries * 2^exp2 */
} otensor;

static int cplx_mode = 1;

static void ot_free(otensor *t) {
    free(t->lab);
    free(t->re);
    free(t->im);
    memset(t, 0, sizeof(*t));
}

static i64 prod_dims(int rank, const int *lab, const i64 *dims) {
    i64 s = 1;
    for (int i = 0; i < rank; ++i) s *= dims[lab[i]];
    return s;
}

/* Row-major strides of tensor t indexed by dense label: stride[l] = 0 if absent. */
static void label_strides(const otensor *t, const i64 *dims, int L, i64 *stride) {
    for (int l = 0; l < L; ++l) stride[l] = 0;
    i64 s = 1;
    for (int i = t->rank - 1; i >= 0; --i) {
        stride[t->lab[i]] = s;
        s *= dims[t->lab[i]];
    }
}

/* Scale by 2^-e where e = frexp exponent of max |component| (Sec. 4.2). */
static void renormalise(otensor *t) {
    double m = 0.0;
    for (i64 i = 0; i < t->size; ++i) {
        double a = fabs(t->re[i]);
        if (a > m) m = a;
        if (t->im) {
            a = fabs(t->im[i]);
            if (a > m) m = a;
        }
    }
    if (m == 0.0) return;
    int e;
    frexp(m, &e);
    if (e == 0) return;
    for (i64 i = 0; i < t->size; ++i) {
        t->re[i] = ldexp(t->re[i], -e);
        if (t->im) t->im[i] = ldexp(t->im[i], -e);
    }
    t->exp2 += e;
}

/*
 * Pairwise contraction (Sec. 2): out[o] = sum_{summed s} A[o,s] * B[o,s]
 * where o runs over the output labels and s over the labels of A or B that
 * are not kept.  A label in both operands and kept is a hyperedge (batch).
 */
static int contract_pair(const otensor *A, const otensor *B, const int *out_lab, int out_rank,
                         const i64 *dims, int L, otensor *C) {
    i64 *sa = (i64 *)malloc(sizeof(i64) * L);
    i64 *sb = (i64 *)malloc(sizeof(i64) * L);
    char *in_out = (char *)calloc(L, 1);
    int *sum_lab = (int *)malloc(sizeof(int) * (A->rank + B->rank + 1));
    if (!sa || !sb || !in_out || !sum_lab) return 2;
    label_strides(A, dims, L, sa);
    label_strides(B, dims, L, sb);
    for (int i = 0; i < out_rank; ++i) in_out[out_lab[i]] = 1;
    int n_sum = 0;
    for (int i = 0; i < A->rank; ++i)
        if (!in_out[A->lab[i]]) sum_lab[n_sum++] = A->lab[i];
    for (int i = 0; i < B->rank; ++i) {
        int l = B->lab[i];
        if (in_out[l]) continue;
        int seen = 0;
        for (int j = 0; j < A->rank; ++j) seen |= (A->lab[j] == l);
        if (!seen) sum_lab[n_sum++] = l;
    }
    C->rank = out_rank;
    C->lab = (int *)malloc(sizeof(int) * (out_rank + 1));
    memcpy(C->lab, out_lab, sizeof(int) * out_rank);
    C->size = prod_dims(out_rank, out_lab, dims);
    C->re = (double *)calloc((size_t)C->size, sizeof(double));
    C->im = cplx_mode ? (double *)calloc((size_t)C->size, sizeof(double)) : NULL;
    C->exp2 = A->exp2 + B->exp2;
    if (!C->lab || !C->re || (cplx_mode && !C->im)) return 2;
    i64 n_sum_entries = prod_dims(n_sum, sum_lab, dims);
    if (n_sum > 64) {
        free(sa);
        free(sb);
        free(in_out);
        free(sum_lab);
        return 1;
    }

    int rc = 0;
#pragma omp parallel for schedule(static) if (C->size >= 1024)
    for (i64 o = 0; o < C->size; ++o) {
        /* decode the output entry into label values (row-major) */
        i64 offa = 0, offb = 0, rem = o;
        for (int i = out_rank - 1; i >= 0; --i) {
            int l = out_lab[i];
            i64 v = rem % dims[l];
            rem /= dims[l];
            offa += v * sa[l];
            offb += v * sb[l];
        }
        int cnt[64];
        for (int i = 0; i < n_sum; ++i) cnt[i] = 0;
        double acc_re = 0.0, acc_im = 0.0;
        i64 ia = offa, ib = offb;
        for (i64 s = 0; s < n_sum_entries; ++s) {
            double ar = A->re[ia], br = B->re[ib];
            if (cplx_mode) {
                double ai = A->im[ia], bi = B->im[ib];
                acc_re += ar * br - ai * bi;
                acc_im += ar * bi + ai * br;
            } else {
                acc_re += ar * br;
            }
            /* odometer over the summed labels, last label fastest */
            for (int i = n_sum - 1; i >= 0; --i) {
                int l = sum_lab[i];
                cnt[i]++;
                ia += sa[l];
                ib += sb[l];
                if (cnt[i] < dims[l]) break;
                ia -= sa[l] * dims[l];
                ib -= sb[l] * dims[l];
                cnt[i] = 0;
            }
        }
        C->re[o] = acc_re;
        if (cplx_mode) C->im[o] = acc_im;
    }
    free(sa);
    free(sb);
    free(in_out);
    free(sum_lab);
    return rc;
}

/* Copy the slice of leaf T with the sliced labels fixed to given values. */
static int slice_leaf(const int rank, const int *lab, const double *data, int is_cplx,
                      const i64 *dims, const i64 *fixed /* -1 if free */, otensor *out) {
    int r = 0;
    out->lab = (int *)malloc(sizeof(int) * (rank + 1));
    for (int i = 0; i < rank; ++i)
        if (fixed[lab[i]] < 0) out->lab[r++] = lab[i];
    out->rank = r;
    out->size = prod_dims(r, out->lab, dims);
    out->re = (double *)malloc(sizeof(double) * (size_t)out->size);
    out->im = is_cplx ? (double *)malloc(sizeof(double) * (size_t)out->size) : NULL;
    out->exp2 = 0;
    if (!out->lab || !out->re || (is_cplx && !out->im)) return 2;
    /* source strides */
    i64 *st = (i64 *)malloc(sizeof(i64) * (rank + 1));
    i64 s = 1;
    for (int i = rank - 1; i >= 0; --i) {
        st[i] = s;
        s *= dims[lab[i]];
    }
    i64 base = 0;
    for (int i = 0; i < rank; ++i)
        if (fixed[lab[i]] >= 0) base += fixed[lab[i]] * st[i];
    for (i64 o = 0; o < out->size; ++o) {
        i64 rem = o, off = base;
        for (int i = rank - 1; i >= 0; --i) {
            if (fixed[lab[i]] >= 0) continue;
            i64 d = dims[lab[i]];
            off += (rem % d) * st[i];
            rem /= d;
        }
        if (is_cplx) {
            out->re[o] = data[2 * off];
            out->im[o] = data[2 * off + 1];
        } else {
            out->re[o] = data[off];
        }
    }
    free(st);
    return 0;
}

static int find_label(int L, const i64 *ids, i64 id) {
    for (int i = 0; i < L; ++i)
        if (ids[i] == id) return i;
    return -1;
}

/*
 * Contract the network with the given tree and sliced labels.
 *   tensors[v]: row-major entries of T_v in the order of its labels; complex
 *               tensors interleave (re, im).
 *   pairs:      2*(n-1) SSA child ids (leaves 0..n-1, node n+i).
 *   slices:     the slice ids slice_begin .. slice_begin+slice_count-1 are
 *               summed (slice id = mixed-radix number of the sliced label
 *               values, last sliced label fastest); slice_count < 0 = all.
 *   out:        n_out entries (complex: interleaved) over the open labels in
 *               the given order; value = out * 2^out_exp2.
 */
int tno_contract(int n_tensors, const int *ranks, const i64 *labels, int n_labels,
                 const i64 *label_ids, const i64 *label_dims, int n_open, const i64 *open_labels,
                 int is_complex, const double *const *tensors, const int *pairs, int n_sliced,
                 const i64 *sliced_labels, i64 slice_begin, i64 slice_count, double *out,
                 i64 *out_exp2) {
    cplx_mode = is_complex ? 1 : 0;
    int L = n_labels;
    int n = n_tensors;
    if (n < 1 || L < 0) return 1;
    i64 *dims = (i64 *)malloc(sizeof(i64) * (L + 1));
    for (int i = 0; i < L; ++i) dims[i] = label_dims[i];
    /* dense label lists of the leaves */
    int **leaf_lab = (int **)malloc(sizeof(int *) * n);
    i64 off = 0;
    for (int v = 0; v < n; ++v) {
        leaf_lab[v] = (int *)malloc(sizeof(int) * (ranks[v] + 1));
        for (int i = 0; i < ranks[v]; ++i) {
            int l = find_label(L, label_ids, labels[off + i]);
            if (l < 0) return 1;
            leaf_lab[v][i] = l;
        }
        off += ranks[v];
    }
    int *open_d = (int *)malloc(sizeof(int) * (n_open + 1));
    char *is_open = (char *)calloc(L + 1, 1);
    for (int i = 0; i < n_open; ++i) {
        open_d[i] = find_label(L, label_ids, open_labels[i]);
        if (open_d[i] < 0) return 1;
        is_open[open_d[i]] = 1;
    }
    int *sl = (int *)malloc(sizeof(int) * (n_sliced + 1));
    i64 d_sliced = 1;
    for (int i = 0; i < n_sliced; ++i) {
        sl[i] = find_label(L, label_ids, sliced_labels[i]);
        if (sl[i] < 0 || is_open[sl[i]]) return 1;
        d_sliced *= dims[sl[i]];
    }
    i64 n_out = prod_dims(n_open, open_d, dims);

    /* total occurrence count of every label over the leaves */
    int *total = (int *)calloc(L + 1, sizeof(int));
    for (int v = 0; v < n; ++v)
        for (int i = 0; i < ranks[v]; ++i) total[leaf_lab[v][i]]++;

    int n_nodes = 2 * n - 1;
    otensor *T = (otensor *)calloc(n_nodes, sizeof(otensor));
    /* per node: count of leaves in the subtree holding each label */
    int **sub = (int **)calloc(n_nodes, sizeof(int *));
    i64 *fixed = (i64 *)malloc(sizeof(i64) * (L + 1));

    double *acc_re = (double *)calloc(n_out, sizeof(double));
    double *acc_im = (double *)calloc(n_out, sizeof(double));
    i64 acc_exp = 0;
    int acc_any = 0;
    int rc = 0;

    i64 s_end = slice_count < 0 ? d_sliced : slice_begin + slice_count;
    if (slice_begin < 0 || s_end > d_sliced) rc = 1;
    for (i64 s = slice_begin; s < s_end && rc == 0; ++s) {
        for (int l = 0; l < L; ++l) fixed[l] = -1;
        i64 rem = s;
        for (int i = n_sliced - 1; i >= 0; --i) {
            fixed[sl[i]] = rem % dims[sl[i]];
            rem /= dims[sl[i]];
        }
        for (int v = 0; v < n; ++v) {
            rc = slice_leaf(ranks[v], leaf_lab[v], tensors[v], is_complex, dims, fixed, &T[v]);
            if (rc) break;
            sub[v] = (int *)calloc(L + 1, sizeof(int));
            for (int i = 0; i < T[v].rank; ++i) sub[v][T[v].lab[i]] = 1;
        }
        /* label totals for this slice ignore the sliced labels (they are gone) */
        for (int k = 0; k < n - 1 && rc == 0; ++k) {
            int a = pairs[2 * k], b = pairs[2 * k + 1], me = n + k;
            sub[me] = (int *)calloc(L + 1, sizeof(int));
            int *outl = (int *)malloc(sizeof(int) * (T[a].rank + T[b].rank + 1));
            int r = 0;
            for (int i = 0; i < T[a].rank; ++i) {
                int l = T[a].lab[i];
                int c = sub[a][l] + sub[b][l];
                sub[me][l] = c;
                if (is_open[l] || c < total[l]) outl[r++] = l;
            }
            for (int i = 0; i < T[b].rank; ++i) {
                int l = T[b].lab[i];
                if (sub[a][l]) continue;
                int c = sub[b][l];
                sub[me][l] = c;
                if (is_open[l] || c < total[l]) outl[r++] = l;
            }
            rc = contract_pair(&T[a], &T[b], outl, r, dims, L, &T[me]);
            free(outl);
            if (rc) break;
            renormalise(&T[me]);
            ot_free(&T[a]);
            ot_free(&T[b]);
        }
        if (rc) break;
        otensor *R = &T[n_nodes - 1];
        if (n == 1) {
            /* a lone tensor: sum out its non-open labels by a pairwise
               contraction with the rank-0 unit tensor */
            otensor one = {0};
            one.size = 1;
            one.re = (double *)malloc(sizeof(double));
            one.re[0] = 1.0;
            if (is_complex) {
                one.im = (double *)malloc(sizeof(double));
                one.im[0] = 0.0;
            }
            one.lab = (int *)malloc(sizeof(int));
            int *outl = (int *)malloc(sizeof(int) * (R->rank + 1));
            int r = 0;
            for (int i = 0; i < R->rank; ++i)
                if (is_open[R->lab[i]]) outl[r++] = R->lab[i];
            otensor red = {0};
            rc = contract_pair(R, &one, outl, r, dims, L, &red);
            free(outl);
            ot_free(&one);
            ot_free(R);
            *R = red;
            if (rc) break;
            renormalise(R);
        }
        if (R->rank != n_open) {
            rc = 1;
            break;
        }
        /* permute the root into the requested open-label order, then
           accumulate into the FP64 result with exponent alignment */
        i64 *rs = (i64 *)malloc(sizeof(i64) * (L + 1));
        label_strides(R, dims, L, rs);
        i64 e_new = R->exp2;
        double f_acc = 1.0, f_new = 1.0;
        if (!acc_any) {
            acc_exp = e_new;
            acc_any = 1;
        } else if (e_new > acc_exp) {
            f_acc = ldexp(1.0, (int)(acc_exp - e_new));
            acc_exp = e_new;
        } else {
            f_new = ldexp(1.0, (int)(e_new - acc_exp));
        }
        for (i64 o = 0; o < n_out; ++o) {
            i64 rr = o, src = 0;
            for (int i = n_open - 1; i >= 0; --i) {
                int l = open_d[i];
                src += (rr % dims[l]) * rs[l];
                rr /= dims[l];
            }
            acc_re[o] = acc_re[o] * f_acc + R->re[src] * f_new;
            if (is_complex) acc_im[o] = acc_im[o] * f_acc + R->im[src] * f_new;
        }
        free(rs);
        ot_free(R);
        for (int v = 0; v < n_nodes; ++v) {
            free(sub[v]);
            sub[v] = NULL;
        }
    }
    if (rc == 0) {
        for (i64 o = 0; o < n_out; ++o) {
            if (is_complex) {
                out[2 * o] = acc_re[o];
                out[2 * o + 1] = acc_im[o];
            } else {
                out[o] = acc_re[o];
            }
        }
        *out_exp2 = acc_exp;
    }
    for (int v = 0; v < n_nodes; ++v) {
        ot_free(&T[v]);
        free(sub[v]);
    }
    for (int v = 0; v < n; ++v) free(leaf_lab[v]);
    free(leaf_lab);
    free(T);
    free(sub);
    free(fixed);
    free(total);
    free(dims);
    free(open_d);
    free(is_open);
    free(sl);
    free(acc_re);
    free(acc_im);
    return rc;
}

int tno_max_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
