/*
 * mps_oracle.c -- plain sequential CPU oracle for Multiway Powersort
 * (Cawley Gelling, Nebel, Smith, Wild: "Multiway Powersort", arXiv 2209.06909).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  It is used by the tests, by the package's smoke check and
 * by the benchmark's CPU-baseline leg, and it shares no code, header, table or
 * helper with the CUDA path.
 *
 * Every function follows the paper's definitions step by step, in the paper's
 * order, with no blocking, fusion or parallel tricks:
 *   - runs: maximal weakly increasing or strictly decreasing segments, found
 *     greedily from the left (Sec. 2 "Preliminaries"; FirstRunOf in Alg. 2);
 *     strictly decreasing runs are reversed before merging (Sec. 2).  An
 *     optional minimum run length (Sec. 5 "Minimal run length", and the
 *     appendix's 4-way Powersort) extends a shorter natural run to that many
 *     elements and insertion-sorts it; 1 keeps the natural runs;
 *   - boundary power: the Power_k procedure of Alg. 2 (equivalently Def. 3.1),
 *     evaluated with exact 128-bit integer floors instead of real division;
 *   - merge policy: the run stack of Alg. 2 (KwayPowerSort_k) with weakly
 *     increasing powers, popping *all* entries of equal top power; the final
 *     collapse applies the same rule against a virtual final power 0, which is
 *     the reading under which Alg. 2 builds the tree of Alg. 1 (Sec. 3.1);
 *   - an independent recursive builder that follows Alg. 1 (KwayTree_k);
 *   - merging: a stable d-way merge (d <= k) that repeatedly outputs the
 *     smallest head, ties going to the leftmost run (the "<=" of the paper's
 *     tournament, Sec. 4 "Tournament tree");
 *   - merge cost M = sum of the sizes of all merge results (Sec. 2.2).
 *
 * Keys are handled as uint64 internally (uint32 inputs are widened); the
 * optional payload is a uint32 per element and moves with its key.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* Node record of the canonical tree encoding (16 bytes). */
typedef struct {
    uint32_t first_run; /* first run (leaf) index covered by the node        */
    uint32_t end_run;   /* one past the last run index covered               */
    uint8_t power;      /* the common power of the node's boundaries         */
    uint8_t degree;     /* number of children d (2 <= d <= k)                */
    uint16_t pad;
    uint32_t parent;    /* index of the parent in the sorted table, or ~0u    */
} mpso_node;

enum { MPSO_OK = 0, MPSO_ERR_ARG = 1, MPSO_ERR_NOMEM = 2, MPSO_ERR_INVARIANT = 3 };

/* ------------------------------------------------------------------------- */
/* Runs (Sec. 2): greedy left-to-right scan.                                  */
/* ------------------------------------------------------------------------- */

/* Finds the end of the leftmost run of a[b..n): if the first two elements are
 * strictly decreasing the run is the maximal strictly decreasing prefix,
 * otherwise the maximal weakly increasing prefix.  *desc is set accordingly. */
static uint64_t first_run_of(const uint64_t* a, uint64_t b, uint64_t n, int* desc) {
    uint64_t e = b + 1;
    if (e < n && a[e] < a[e - 1]) {
        while (e < n && a[e] < a[e - 1]) e++;
        *desc = 1;
    } else {
        while (e < n && a[e] >= a[e - 1]) e++;
        *desc = 0;
    }
    return e;
}

/* Runs with a minimum length min_run_len >= 1: the natural run found from b
 * (FirstRunOf) ends the run unless it is shorter than min_run_len, in which
 * case the run takes min(n, b + min_run_len) elements (Sec. 5 "Minimal run
 * length").  The next run is searched from the end of this one in the input
 * as given.  Writes run starts s_0..s_{r-1}, s_r = n, the direction of each
 * run's natural part and, if nat_len is not NULL, that part's length;
 * returns r. */
uint64_t mpso_find_runs_min(const uint64_t* a, uint64_t n, uint32_t min_run_len, uint32_t* starts, uint8_t* desc,
                            uint32_t* nat_len) {
    uint64_t r = 0, b = 0;
    if (min_run_len < 1) min_run_len = 1;
    while (b < n) {
        int d = 0;
        uint64_t e = first_run_of(a, b, n, &d);
        const uint64_t natural = e - b;
        if (natural < min_run_len) e = (n - b > min_run_len) ? b + min_run_len : n;
        starts[r] = (uint32_t)b;
        desc[r] = (uint8_t)d;
        if (nat_len) nat_len[r] = (uint32_t)natural;
        r++;
        b = e;
    }
    starts[r] = (uint32_t)n;
    return r;
}

/* Natural runs: writes run starts s_0..s_{r-1}, s_r = n and direction flags;
 * returns r. */
uint64_t mpso_find_runs(const uint64_t* a, uint64_t n, uint32_t* starts, uint8_t* desc) {
    return mpso_find_runs_min(a, n, 1, starts, desc, NULL);
}

/* ------------------------------------------------------------------------- */
/* Power_k (Alg. 2, procedure Power_k; Def. 3.1).                             */
/* ------------------------------------------------------------------------- */

/* a = (b1 + n1/2)/n and b = (b2 + n2/2)/n are the normalised midpoints of the
 * two runs; p is the smallest non-negative integer with
 * floor(a k^p) != floor(b k^p).  With a = (2 b1 + n1) / (2n) every floor is an
 * exact integer quotient.  The loop stops by p <= ceil(log_k n) + 1 (the
 * paper's bound on powers), far below the 128-bit limit for n < 2^32. */
uint32_t mpso_power(uint64_t n, uint64_t b1, uint64_t e1, uint64_t b2, uint64_t e2, uint32_t k) {
    uint64_t n1 = e1 - b1, n2 = e2 - b2;
    u128 num_a = (u128)(2 * b1 + n1);
    u128 num_b = (u128)(2 * b2 + n2);
    u128 den = (u128)(2 * n);
    u128 kp = 1;
    uint32_t p = 0;
    while ((num_a * kp) / den == (num_b * kp) / den) {
        p++;
        kp *= k;
        if (p > 100) return 0xFFFFFFFFu; /* unreachable for valid runs */
    }
    return p;
}

/* ------------------------------------------------------------------------- */
/* Raw tree bookkeeping shared by the two builders below.                     */
/* ------------------------------------------------------------------------- */

typedef struct {
    uint32_t first_run, end_run, power, degree;
    int64_t parent;   /* raw id, -1 for the root */
    uint32_t min_boundary;
} raw_node;

typedef struct {
    raw_node* v;
    uint64_t count, cap;
    int64_t* boundary_node; /* raw node id owning boundary i (1..r-1) */
    int64_t* leaf_parent;   /* raw node id of the parent of run i, -1 if none */
} raw_tree;

static int raw_tree_init(raw_tree* t, uint64_t r) {
    t->cap = r > 1 ? r - 1 : 1;
    t->count = 0;
    t->v = (raw_node*)calloc(t->cap, sizeof(raw_node));
    t->boundary_node = (int64_t*)malloc((r + 1) * sizeof(int64_t));
    t->leaf_parent = (int64_t*)malloc((r + 1) * sizeof(int64_t));
    if (!t->v || !t->boundary_node || !t->leaf_parent) return MPSO_ERR_NOMEM;
    for (uint64_t i = 0; i <= r; i++) { t->boundary_node[i] = -1; t->leaf_parent[i] = -1; }
    return MPSO_OK;
}

static void raw_tree_free(raw_tree* t) {
    free(t->v); free(t->boundary_node); free(t->leaf_parent);
}

/* Sorting helpers for the canonical order (power, first_run). */
static const raw_node* g_sort_nodes;
static int cmp_canon(const void* x, const void* y) {
    const raw_node* a = &g_sort_nodes[*(const uint64_t*)x];
    const raw_node* b = &g_sort_nodes[*(const uint64_t*)y];
    if (a->power != b->power) return a->power < b->power ? -1 : 1;
    if (a->first_run != b->first_run) return a->first_run < b->first_run ? -1 : 1;
    return 0;
}

/* Emits the canonical encoding: node table sorted by (power, first_run),
 * node_first[i] = smallest boundary of the node owning boundary i,
 * leaf_depth[i] = edges from run i to the root, and M = sum of node sizes
 * (Sec. 2.2), cross-checked against sum_i d_i L_i. */
static int emit_canonical(const raw_tree* t, const uint32_t* starts, uint64_t r,
                          mpso_node* nodes, uint32_t* node_first, uint8_t* leaf_depth,
                          uint64_t* counts) {
    uint64_t m = t->count;
    uint64_t* order = (uint64_t*)malloc((m ? m : 1) * sizeof(uint64_t));
    uint64_t* rank = (uint64_t*)malloc((m ? m : 1) * sizeof(uint64_t));
    int64_t* depth = (int64_t*)malloc((m ? m : 1) * sizeof(int64_t));
    if (!order || !rank || !depth) { free(order); free(rank); free(depth); return MPSO_ERR_NOMEM; }
    for (uint64_t i = 0; i < m; i++) order[i] = i;
    g_sort_nodes = t->v;
    qsort(order, m, sizeof(uint64_t), cmp_canon);
    for (uint64_t i = 0; i < m; i++) rank[order[i]] = i;

    /* node depth by walking parent links (root depth 0) */
    for (uint64_t i = 0; i < m; i++) {
        int64_t d = 0, u = t->v[i].parent;
        while (u >= 0) { d++; u = t->v[u].parent; }
        depth[i] = d;
    }
    uint64_t merge_cost = 0, distinct = 0, seen[256] = {0};
    for (uint64_t i = 0; i < m; i++) {
        const raw_node* v = &t->v[order[i]];
        if (nodes) {
            nodes[i].first_run = v->first_run;
            nodes[i].end_run = v->end_run;
            nodes[i].power = (uint8_t)v->power;
            nodes[i].degree = (uint8_t)v->degree;
            nodes[i].pad = 0;
            nodes[i].parent = v->parent < 0 ? 0xFFFFFFFFu : (uint32_t)rank[v->parent];
        }
        merge_cost += (uint64_t)starts[v->end_run] - starts[v->first_run];
        if (!seen[v->power & 255]) { seen[v->power & 255] = 1; distinct++; }
    }
    if (node_first) {
        node_first[0] = 0;
        for (uint64_t i = 1; i < r; i++) node_first[i] = t->v[t->boundary_node[i]].min_boundary;
    }
    uint64_t sum_dl = 0;
    for (uint64_t i = 0; i < r; i++) {
        int64_t p = t->leaf_parent[i];
        uint64_t d = p < 0 ? 0 : (uint64_t)depth[p] + 1;
        if (leaf_depth) leaf_depth[i] = (uint8_t)d;
        sum_dl += d * ((uint64_t)starts[i + 1] - starts[i]);
    }
    free(order); free(rank); free(depth);
    if (counts) { counts[0] = r; counts[1] = m; counts[2] = distinct; counts[3] = merge_cost; }
    return sum_dl == merge_cost ? MPSO_OK : MPSO_ERR_INVARIANT;
}

/* ------------------------------------------------------------------------- */
/* Stable d-way merge of adjacent sorted segments (Sec. 2.2, Sec. 4).          */
/* ------------------------------------------------------------------------- */

/* Segments seg[0..d] delimit d adjacent sorted runs of a[seg[0]..seg[d]).
 * Copies them to the buffer and repeatedly outputs the smallest head; on
 * equal keys the leftmost run wins, which keeps the merge stable. */
static void merge_segments(uint64_t* a, uint32_t* v, uint64_t* buf, uint32_t* vbuf,
                           const uint64_t* seg, uint32_t d) {
    uint64_t lo = seg[0], hi = seg[d];
    memcpy(buf, a + lo, (hi - lo) * sizeof(uint64_t));
    if (v) memcpy(vbuf, v + lo, (hi - lo) * sizeof(uint32_t));
    uint64_t head[64], end[64];
    for (uint32_t c = 0; c < d; c++) { head[c] = seg[c] - lo; end[c] = seg[c + 1] - lo; }
    for (uint64_t o = lo; o < hi; o++) {
        int best = -1;
        for (uint32_t c = 0; c < d; c++) {
            if (head[c] == end[c]) continue;
            if (best < 0 || buf[head[c]] < buf[head[best]]) best = (int)c;
        }
        a[o] = buf[head[best]];
        if (v) v[o] = vbuf[head[best]];
        head[best]++;
    }
}

/* ------------------------------------------------------------------------- */
/* Alg. 2: KwayPowerSort_k with the run stack.                                */
/* ------------------------------------------------------------------------- */

typedef struct {
    uint64_t b, e;          /* element range of the (merged) segment */
    uint32_t first_run, end_run;
    int64_t node;           /* raw node id, -1 for a single run       */
    uint32_t power;         /* power of the boundary at its right end  */
    uint32_t boundary;      /* index of that boundary                  */
} stack_entry;

/* Merges every stack entry whose power equals the top power with the current
 * segment *cur, records the resulting node, and returns the new segment. */
static int collapse_top(stack_entry* st, uint64_t* sp, stack_entry* cur, raw_tree* t,
                        uint64_t* a, uint32_t* vals, uint64_t* buf, uint32_t* vbuf, uint32_t k) {
    uint32_t ptop = st[*sp - 1].power;
    uint64_t cnt = 0;
    while (*sp > 0 && st[*sp - 1].power == ptop) { (*sp)--; cnt++; }
    if (cnt + 1 > k || cnt + 1 > 64) return MPSO_ERR_INVARIANT;
    /* children in left-to-right order: st[*sp .. *sp+cnt), then *cur */
    uint64_t seg[65];
    uint32_t d = (uint32_t)cnt + 1;
    for (uint64_t c = 0; c < cnt; c++) seg[c] = st[*sp + c].b;
    seg[cnt] = cur->b;
    seg[cnt + 1] = cur->e;
    if (a) merge_segments(a, vals, buf, vbuf, seg, d);

    uint64_t id = t->count++;
    raw_node* nv = &t->v[id];
    nv->first_run = st[*sp].first_run;
    nv->end_run = cur->end_run;
    nv->power = ptop;
    nv->degree = d;
    nv->parent = -1;
    nv->min_boundary = st[*sp].boundary;
    for (uint64_t c = 0; c < cnt; c++) {
        const stack_entry* ch = &st[*sp + c];
        t->boundary_node[ch->boundary] = (int64_t)id;
        if (ch->node >= 0) t->v[ch->node].parent = (int64_t)id;
        else t->leaf_parent[ch->first_run] = (int64_t)id;
    }
    if (cur->node >= 0) t->v[cur->node].parent = (int64_t)id;
    else t->leaf_parent[cur->first_run] = (int64_t)id;

    cur->b = st[*sp].b;
    cur->first_run = st[*sp].first_run;
    cur->node = (int64_t)id;
    return MPSO_OK;
}

/*
 * Sorts keys with Multiway Powersort and reports the run structure and tree.
 *   keys_in/keys_out : n keys of key_bytes (4 or 8) bytes; may alias.
 *   vals_in/vals_out : optional uint32 payload (both NULL or both set).
 *   k                : fan-in, k >= 2.
 *   min_run_len      : minimum run length (>= 1; 1 = natural runs); run_desc
 *                      then flags a strictly decreasing natural part.
 *   run_starts[r+1], run_desc[r], powers[r+1] (powers[0]=powers[r]=0),
 *   nodes[r-1], node_first[r], leaf_depth[r], counts[4] = {r, nodes, levels, M}:
 *   optional outputs (NULL to skip), sized for the worst case r = n.
 */
int mpso_sort_min_run(const void* keys_in, const uint32_t* vals_in, void* keys_out, uint32_t* vals_out,
                      uint64_t n, int key_bytes, uint32_t k, uint32_t min_run_len,
                      uint32_t* run_starts, uint8_t* run_desc, uint8_t* powers,
                      mpso_node* nodes, uint32_t* node_first, uint8_t* leaf_depth, uint64_t* counts) {
    if ((key_bytes != 4 && key_bytes != 8) || k < 2 || n >= (1ull << 32) || min_run_len < 1) return MPSO_ERR_ARG;
    if ((vals_in == NULL) != (vals_out == NULL)) return MPSO_ERR_ARG;
    int rc = MPSO_OK;
    uint64_t* a = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    uint64_t* buf = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    uint32_t* v = vals_in ? (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t)) : NULL;
    uint32_t* vbuf = vals_in ? (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t)) : NULL;
    uint32_t* st_s = (uint32_t*)malloc((n + 2) * sizeof(uint32_t));
    uint8_t* st_d = (uint8_t*)malloc(n + 2);
    uint32_t* st_l = (uint32_t*)malloc((n + 2) * sizeof(uint32_t));
    if (!a || !buf || !st_s || !st_d || !st_l || (vals_in && (!v || !vbuf))) { rc = MPSO_ERR_NOMEM; goto done0; }
    for (uint64_t i = 0; i < n; i++)
        a[i] = key_bytes == 4 ? ((const uint32_t*)keys_in)[i] : ((const uint64_t*)keys_in)[i];
    if (v) memcpy(v, vals_in, n * sizeof(uint32_t));

    /* runs, then reverse the strictly decreasing natural parts (stable: no
     * ties) and insertion-sort each extended run; its first natural-length
     * elements are sorted already, and an element moves left only past
     * strictly larger keys, so equal keys keep their order */
    uint64_t r = mpso_find_runs_min(a, n, min_run_len, st_s, st_d, st_l);
    for (uint64_t i = 0; i < r; i++) {
        const uint64_t s0 = st_s[i], s1 = st_s[i + 1], nat = st_l[i];
        if (st_d[i]) {
            uint64_t lo = s0, hi = s0 + nat - 1;
            while (lo < hi) {
                uint64_t tk = a[lo]; a[lo] = a[hi]; a[hi] = tk;
                if (v) { uint32_t tv = v[lo]; v[lo] = v[hi]; v[hi] = tv; }
                lo++; hi--;
            }
        }
        for (uint64_t x = s0 + nat; x < s1; x++) {
            const uint64_t key = a[x];
            const uint32_t val = v ? v[x] : 0u;
            uint64_t y = x;
            while (y > s0 && a[y - 1] > key) {
                a[y] = a[y - 1];
                if (v) v[y] = v[y - 1];
                y--;
            }
            a[y] = key;
            if (v) v[y] = val;
        }
    }

    raw_tree t;
    if ((rc = raw_tree_init(&t, r)) != MPSO_OK) { raw_tree_free(&t); goto done0; }
    uint8_t* pw = (uint8_t*)calloc(r + 1, 1);
    /* stack capacity (k-1) * ceil(log_k n + 1) (Sec. 3.3); a generous bound */
    stack_entry* st = (stack_entry*)malloc((64 * (uint64_t)k + 8) * sizeof(stack_entry));
    if (!pw || !st) { rc = MPSO_ERR_NOMEM; goto done1; }

    uint64_t sp = 0;
    if (r > 0) {
        stack_entry cur = {st_s[0], st_s[1], 0, 1, -1, 0, 0};
        for (uint64_t i = 1; i < r; i++) {
            /* next run (b2, e2) = run i; power of boundary i between run i-1 and run i */
            uint32_t P = mpso_power(n, st_s[i - 1], st_s[i], st_s[i], st_s[i + 1], k);
            pw[i] = (uint8_t)P;
            while (sp > 0 && st[sp - 1].power > P)
                if ((rc = collapse_top(st, &sp, &cur, &t, a, v, buf, vbuf, k)) != MPSO_OK) goto done1;
            cur.power = P;
            cur.boundary = (uint32_t)i;
            if (sp >= 64 * (uint64_t)k + 8) { rc = MPSO_ERR_INVARIANT; goto done1; }
            st[sp++] = cur;
            stack_entry nxt = {st_s[i], st_s[i + 1], (uint32_t)i, (uint32_t)i + 1, -1, 0, 0};
            cur = nxt;
        }
        /* final collapse: the same power rule against a virtual final power 0 */
        while (sp > 0)
            if ((rc = collapse_top(st, &sp, &cur, &t, a, v, buf, vbuf, k)) != MPSO_OK) goto done1;
    }

    for (uint64_t i = 0; i < n; i++) {
        if (key_bytes == 4) ((uint32_t*)keys_out)[i] = (uint32_t)a[i];
        else ((uint64_t*)keys_out)[i] = a[i];
    }
    if (vals_out) memcpy(vals_out, v, n * sizeof(uint32_t));
    if (run_starts) memcpy(run_starts, st_s, (r + 1) * sizeof(uint32_t));
    if (run_desc) memcpy(run_desc, st_d, r);
    if (powers) { memcpy(powers, pw, r + 1); powers[0] = 0; if (r > 0) powers[r] = 0; }
    rc = emit_canonical(&t, st_s, r, nodes, node_first, leaf_depth, counts);

done1:
    free(pw); free(st);
    raw_tree_free(&t);
done0:
    free(a); free(buf); free(v); free(vbuf); free(st_s); free(st_d); free(st_l);
    return rc;
}

/* Multiway Powersort on natural runs (minimum run length 1). */
int mpso_sort(const void* keys_in, const uint32_t* vals_in, void* keys_out, uint32_t* vals_out,
              uint64_t n, int key_bytes, uint32_t k,
              uint32_t* run_starts, uint8_t* run_desc, uint8_t* powers,
              mpso_node* nodes, uint32_t* node_first, uint8_t* leaf_depth, uint64_t* counts) {
    return mpso_sort_min_run(keys_in, vals_in, keys_out, vals_out, n, key_bytes, k, 1, run_starts, run_desc, powers,
                             nodes, node_first, leaf_depth, counts);
}

/* ------------------------------------------------------------------------- */
/* Alg. 1: KwayTree_k, the recursive conceptual builder.                      */
/* ------------------------------------------------------------------------- */

/* Builds the subtree over runs [lo, hi) (hi - lo >= 2) by splitting at every
 * boundary of minimum power; returns its raw node id. */
static int64_t kway_tree_rec(const uint8_t* pw, uint64_t lo, uint64_t hi, raw_tree* t, int* err) {
    uint32_t pmin = 0xFFFFFFFFu;
    for (uint64_t i = lo + 1; i < hi; i++) if (pw[i] < pmin) pmin = pw[i];
    uint64_t id = t->count++;
    raw_node* nv = &t->v[id];
    nv->first_run = (uint32_t)lo;
    nv->end_run = (uint32_t)hi;
    nv->power = pmin;
    nv->parent = -1;
    uint32_t d = 1;
    uint64_t piece = lo;
    nv->min_boundary = 0;
    for (uint64_t i = lo + 1; i <= hi; i++) {
        if (i < hi && pw[i] != pmin) continue;
        if (i < hi) {
            t->boundary_node[i] = (int64_t)id;
            if (d == 1) t->v[id].min_boundary = (uint32_t)i;
            d++;
        }
        /* child piece [piece, i) */
        if (i - piece >= 2) {
            int64_t c = kway_tree_rec(pw, piece, i, t, err);
            t->v[c].parent = (int64_t)id;
        } else {
            t->leaf_parent[piece] = (int64_t)id;
        }
        piece = i;
    }
    t->v[id].degree = d;
    return (int64_t)id;
}

/* Tree of Alg. 1 from a powers array (powers[1..r-1]) and run starts. */
int mpso_tree_from_powers(const uint8_t* powers, const uint32_t* run_starts, uint64_t r,
                          mpso_node* nodes, uint32_t* node_first, uint8_t* leaf_depth, uint64_t* counts) {
    raw_tree t;
    int rc = raw_tree_init(&t, r);
    if (rc == MPSO_OK) {
        int err = 0;
        if (r >= 2) kway_tree_rec(powers, 0, r, &t, &err);
        rc = err ? MPSO_ERR_INVARIANT : emit_canonical(&t, run_starts, r, nodes, node_first, leaf_depth, counts);
    }
    raw_tree_free(&t);
    return rc;
}

/* Powers (Alg. 2's Power_k) for a vector of run lengths; powers[0] = powers[r] = 0. */
int mpso_powers_from_lengths(const uint64_t* lengths, uint64_t r, uint32_t k, uint8_t* powers,
                             uint32_t* run_starts) {
    uint64_t s = 0;
    for (uint64_t i = 0; i < r; i++) { run_starts[i] = (uint32_t)s; s += lengths[i]; }
    run_starts[r] = (uint32_t)s;
    powers[0] = 0;
    for (uint64_t i = 1; i < r; i++)
        powers[i] = (uint8_t)mpso_power(s, run_starts[i - 1], run_starts[i], run_starts[i], run_starts[i + 1], k);
    if (r > 0) powers[r] = 0;
    return MPSO_OK;
}

/* Runs the stack policy of Alg. 2 on run lengths alone (no data movement):
 * returns the canonical tree for the given lengths. */
int mpso_tree_from_lengths(const uint64_t* lengths, uint64_t r, uint32_t k,
                           mpso_node* nodes, uint32_t* node_first, uint8_t* leaf_depth, uint64_t* counts,
                           uint8_t* powers_out) {
    uint32_t* starts = (uint32_t*)malloc((r + 1) * sizeof(uint32_t));
    uint8_t* pw = (uint8_t*)calloc(r + 1, 1);
    stack_entry* st = (stack_entry*)malloc((64 * (uint64_t)k + 8) * sizeof(stack_entry));
    raw_tree t;
    int rc = raw_tree_init(&t, r);
    if (!starts || !pw || !st || rc != MPSO_OK) { rc = MPSO_ERR_NOMEM; goto out; }
    mpso_powers_from_lengths(lengths, r, k, pw, starts);
    uint64_t sp = 0;
    if (r > 0) {
        stack_entry cur = {starts[0], starts[1], 0, 1, -1, 0, 0};
        for (uint64_t i = 1; i < r; i++) {
            uint32_t P = pw[i];
            while (sp > 0 && st[sp - 1].power > P)
                if ((rc = collapse_top(st, &sp, &cur, &t, NULL, NULL, NULL, NULL, k)) != MPSO_OK) goto out;
            cur.power = P;
            cur.boundary = (uint32_t)i;
            if (sp >= 64 * (uint64_t)k + 8) { rc = MPSO_ERR_INVARIANT; goto out; }
            st[sp++] = cur;
            stack_entry nxt = {starts[i], starts[i + 1], (uint32_t)i, (uint32_t)i + 1, -1, 0, 0};
            cur = nxt;
        }
        while (sp > 0)
            if ((rc = collapse_top(st, &sp, &cur, &t, NULL, NULL, NULL, NULL, k)) != MPSO_OK) goto out;
    }
    if (powers_out) memcpy(powers_out, pw, r + 1);
    rc = emit_canonical(&t, starts, r, nodes, node_first, leaf_depth, counts);
out:
    free(starts); free(pw); free(st);
    raw_tree_free(&t);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Final-collapse variants: the full tree.                                    */
/* ------------------------------------------------------------------------- */

/* Pops exactly cnt stack entries, whatever their powers, and merges them with
 * the current segment *cur into one node (the last loop of Alg. 2 and the
 * appendix's merge_down pop by count, not by power).  The node's power label
 * is the smallest power among its boundaries, which is the power of the
 * lowest popped entry (powers never decrease up the stack). */
static int collapse_count(stack_entry* st, uint64_t* sp, stack_entry* cur, raw_tree* t, uint64_t cnt, uint32_t k) {
    if (cnt == 0 || cnt > *sp || cnt + 1 > k || cnt + 1 > 64) return MPSO_ERR_INVARIANT;
    *sp -= cnt;
    const uint64_t id = t->count++;
    raw_node* nv = &t->v[id];
    nv->first_run = st[*sp].first_run;
    nv->end_run = cur->end_run;
    nv->power = st[*sp].power;
    nv->degree = (uint32_t)cnt + 1;
    nv->parent = -1;
    nv->min_boundary = st[*sp].boundary;
    for (uint64_t c = 0; c < cnt; c++) {
        const stack_entry* ch = &st[*sp + c];
        t->boundary_node[ch->boundary] = (int64_t)id;
        if (ch->node >= 0) t->v[ch->node].parent = (int64_t)id;
        else t->leaf_parent[ch->first_run] = (int64_t)id;
    }
    if (cur->node >= 0) t->v[cur->node].parent = (int64_t)id;
    else t->leaf_parent[cur->first_run] = (int64_t)id;
    cur->b = st[*sp].b;
    cur->first_run = st[*sp].first_run;
    cur->node = (int64_t)id;
    return MPSO_OK;
}

/*
 * The tree that Alg. 2's run stack builds on run lengths alone when the stack
 * left after the last run is emptied by `policy` (0, 1 or 2 as for
 * mpso_merge_cost_tail below); the main loop is Alg. 2's in all three.  The
 * nodes made by the main loop carry the power of their boundaries; a node of
 * the final collapse under policy 1 or 2 carries the smallest power among its
 * boundaries (its children need not share one).  Outputs as for
 * mpso_tree_from_lengths (canonical order (power label, first run)).
 */
int mpso_tree_tail(const uint64_t* lengths, uint64_t r, uint32_t k, int policy,
                   mpso_node* nodes, uint32_t* node_first, uint8_t* leaf_depth, uint64_t* counts) {
    if (k < 2 || policy < 0 || policy > 2) return MPSO_ERR_ARG;
    uint32_t* starts = (uint32_t*)malloc((r + 1) * sizeof(uint32_t));
    uint8_t* pw = (uint8_t*)calloc(r + 1, 1);
    stack_entry* st = (stack_entry*)malloc((64 * (uint64_t)k + 8) * sizeof(stack_entry));
    raw_tree t;
    int rc = raw_tree_init(&t, r);
    if (!starts || !pw || !st || rc != MPSO_OK) { rc = MPSO_ERR_NOMEM; goto out; }
    mpso_powers_from_lengths(lengths, r, k, pw, starts);
    uint64_t sp = 0;
    if (r > 0) {
        stack_entry cur = {starts[0], starts[1], 0, 1, -1, 0, 0};
        for (uint64_t i = 1; i < r; i++) {
            const uint32_t P = pw[i];
            while (sp > 0 && st[sp - 1].power > P)
                if ((rc = collapse_top(st, &sp, &cur, &t, NULL, NULL, NULL, NULL, k)) != MPSO_OK) goto out;
            cur.power = P;
            cur.boundary = (uint32_t)i;
            if (sp >= 64 * (uint64_t)k + 8) { rc = MPSO_ERR_INVARIANT; goto out; }
            st[sp++] = cur;
            stack_entry nxt = {starts[i], starts[i + 1], (uint32_t)i, (uint32_t)i + 1, -1, 0, 0};
            cur = nxt;
        }
        if (policy == 0) {
            while (sp > 0)
                if ((rc = collapse_top(st, &sp, &cur, &t, NULL, NULL, NULL, NULL, k)) != MPSO_OK) goto out;
        } else {
            /* policy 2 first merges x = (entries) mod (k - 1) entries, so that
             * every later node has k children; policy 1 takes k - 1 each time */
            const uint64_t x = policy == 2 ? sp % (k - 1) : 0;
            if (x > 0 && (rc = collapse_count(st, &sp, &cur, &t, x, k)) != MPSO_OK) goto out;
            while (sp > 0) {
                const uint64_t cnt = sp < (uint64_t)(k - 1) ? sp : (uint64_t)(k - 1);
                if ((rc = collapse_count(st, &sp, &cur, &t, cnt, k)) != MPSO_OK) goto out;
            }
        }
    }
    rc = emit_canonical(&t, starts, r, nodes, node_first, leaf_depth, counts);
out:
    free(starts); free(pw); free(st);
    raw_tree_free(&t);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Final-collapse variants (merge cost only).                                 */
/* ------------------------------------------------------------------------- */

/*
 * Merge cost of Alg. 2's run stack on run lengths alone, with one of three
 * ways to empty the stack after the last run (the main loop is the same in
 * all three: while the top power exceeds the new boundary's power, merge the
 * group of equal top powers with the current run):
 *   policy 0: the same power rule against a virtual final power 0 -- the tree
 *             of Alg. 1 (KwayTree_k), as everywhere else in this oracle;
 *   policy 1: Alg. 2's last loop as printed: pop up to k-1 runs at a time and
 *             merge them with the current run;
 *   policy 2: the appendix's merge_down for k = 4, taken to any k: first merge
 *             the top x runs with the current run, x = (runs - 1) mod (k - 1),
 *             so that every later merge takes k runs (k-1 popped + current).
 * *cost receives M = the sum of the sizes of all merge results (Sec. 2.2).
 */
int mpso_merge_cost_tail(const uint64_t* lengths, uint64_t r, uint32_t k, int policy, uint64_t* cost) {
    if (k < 2 || policy < 0 || policy > 2 || !cost) return MPSO_ERR_ARG;
    *cost = 0;
    if (r <= 1) return MPSO_OK;
    uint32_t* starts = (uint32_t*)malloc((r + 1) * sizeof(uint32_t));
    uint8_t* pw = (uint8_t*)calloc(r + 1, 1);
    uint64_t* sl = (uint64_t*)malloc((r + 1) * sizeof(uint64_t)); /* stack: lengths */
    uint32_t* sp_pw = (uint32_t*)malloc((r + 1) * sizeof(uint32_t)); /* stack: powers */
    if (!starts || !pw || !sl || !sp_pw) {
        free(starts); free(pw); free(sl); free(sp_pw);
        return MPSO_ERR_NOMEM;
    }
    mpso_powers_from_lengths(lengths, r, k, pw, starts);
    uint64_t sp = 0, cur = lengths[0], m = 0;
    for (uint64_t i = 1; i < r; i++) {
        const uint32_t P = pw[i];
        while (sp > 0 && sp_pw[sp - 1] > P) {
            const uint32_t top = sp_pw[sp - 1];
            while (sp > 0 && sp_pw[sp - 1] == top) cur += sl[--sp];
            m += cur;
        }
        sl[sp] = cur;
        sp_pw[sp] = P;
        sp++;
        cur = lengths[i];
    }
    if (policy == 0) {
        while (sp > 0) {
            const uint32_t top = sp_pw[sp - 1];
            while (sp > 0 && sp_pw[sp - 1] == top) cur += sl[--sp];
            m += cur;
        }
    } else if (policy == 1) {
        while (sp > 0) {
            for (uint32_t c = 0; c + 1 < k && sp > 0; c++) cur += sl[--sp];
            m += cur;
        }
    } else {
        const uint64_t x = sp % (k - 1); /* (stack + current - 1) mod (k - 1) */
        if (x > 0) {
            for (uint64_t c = 0; c < x; c++) cur += sl[--sp];
            m += cur;
        }
        while (sp > 0) {
            for (uint32_t c = 0; c + 1 < k; c++) cur += sl[--sp];
            m += cur;
        }
    }
    *cost = m;
    free(starts); free(pw); free(sl); free(sp_pw);
    return MPSO_OK;
}
