/*
 * Oracle for exact multiple pattern matching -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, the smoke check and the CPU-baseline leg of bench.py load this
 * library.  It shares no code, header, table or helper with the CUDA library;
 * it is a plain, slow, obviously correct restatement of what the search must
 * return.
 *
 * Problem statement (Section 1, "Introduction"): given a text T of length n
 * and a set of r patterns P_1..P_r, each of length m, over a common alphabet,
 * report every occurrence.  An occurrence is a pair (i, p) with
 * T[i..i+m) == P_p.  Output order (the paper fixes none): ascending position
 * i, then ascending pattern id p (0-based); identical patterns are each
 * reported.
 *
 * Two independent implementations:
 *   oracle_naive      -- r x n direct comparison with early exit.
 *   oracle_ac_*       -- textbook Aho-Corasick automaton (Section 1.1: a
 *                        pattern trie with failure links, O(M + n + z)),
 *                        byte alphabet, child lists, BFS failure links and
 *                        dictionary-suffix (output) links.  The threaded
 *                        search splits the START positions into contiguous
 *                        ranges; each range is scanned from the root over
 *                        [a, b + m - 1) and reports only starts in [a, b),
 *                        so every occurrence is reported exactly once and the
 *                        concatenation in range order is sorted.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------ naive */

/* Returns the total number of occurrences; writes at most `cap` of them. */
int64_t oracle_naive(const uint8_t *T, uint64_t n, const uint8_t *P,
                     uint64_t r, uint64_t m, uint32_t *out_pos,
                     uint32_t *out_pid, uint64_t cap)
{
    int64_t z = 0;
    if (m == 0 || n < m) return 0;
    for (uint64_t i = 0; i + m <= n; i++) {
        for (uint64_t p = 0; p < r; p++) {
            const uint8_t *pat = P + p * m;
            uint64_t j = 0;
            while (j < m && T[i + j] == pat[j]) j++;
            if (j == m) {
                if ((uint64_t)z < cap) {
                    out_pos[z] = (uint32_t)i;
                    out_pid[z] = (uint32_t)p;
                }
                z++;
            }
        }
    }
    return z;
}

/* ----------------------------------------------------------- Aho-Corasick */

typedef struct {
    int32_t first_child;   /* head of the child list, -1 if none          */
    int32_t next_sibling;  /* next node in the parent's child list        */
    int32_t fail;          /* failure link                                */
    int32_t out;           /* nearest proper-suffix node ending a pattern */
    int32_t pid_head;      /* first pattern id ending exactly here, -1    */
    int32_t depth;
    uint8_t label;         /* edge label from the parent                  */
} ac_node;

typedef struct {
    ac_node *nodes;
    int32_t nnodes, cap;
    int32_t *pid_next;     /* pattern ids ending at the same node, a list */
    uint64_t r, m;         /* m: the longest pattern                      */
    uint64_t mmin;         /* the shortest pattern                        */
} ac_automaton;

static int32_t ac_child(const ac_automaton *a, int32_t v, uint8_t c)
{
    for (int32_t u = a->nodes[v].first_child; u >= 0; u = a->nodes[u].next_sibling)
        if (a->nodes[u].label == c) return u;
    return -1;
}

static int32_t ac_new_node(ac_automaton *a, uint8_t label, int32_t depth)
{
    if (a->nnodes == a->cap) {
        int32_t ncap = a->cap ? a->cap * 2 : 1024;
        ac_node *nn = (ac_node *)realloc(a->nodes, sizeof(ac_node) * (size_t)ncap);
        if (!nn) return -1;
        a->nodes = nn;
        a->cap = ncap;
    }
    ac_node *x = &a->nodes[a->nnodes];
    x->first_child = -1;
    x->next_sibling = -1;
    x->fail = 0;
    x->out = -1;
    x->pid_head = -1;
    x->depth = depth;
    x->label = label;
    return a->nnodes++;
}

void oracle_ac_free(void *h)
{
    ac_automaton *a = (ac_automaton *)h;
    if (!a) return;
    free(a->nodes);
    free(a->pid_next);
    free(a);
}

/* Builds the automaton for r patterns; pattern p is P[off[p] .. off[p+1]). */
void *oracle_ac_build_var(const uint8_t *P, const uint64_t *off, uint64_t r)
{
    ac_automaton *a = (ac_automaton *)calloc(1, sizeof(ac_automaton));
    if (!a) return NULL;
    a->r = r;
    a->m = 0;
    a->mmin = r ? (uint64_t)-1 : 0;
    for (uint64_t p = 0; p < r; p++) {
        const uint64_t len = off[p + 1] - off[p];
        if (len > a->m) a->m = len;
        if (len < a->mmin) a->mmin = len;
    }
    a->pid_next = (int32_t *)malloc(sizeof(int32_t) * (r ? r : 1));
    if (!a->pid_next || ac_new_node(a, 0, 0) < 0) { oracle_ac_free(a); return NULL; }

    /* 1. the trie of all patterns */
    int32_t *pid_tail = NULL;
    for (uint64_t p = 0; p < r; p++) {
        int32_t v = 0;
        const uint64_t len = off[p + 1] - off[p];
        for (uint64_t j = 0; j < len; j++) {
            uint8_t c = P[off[p] + j];
            int32_t u = ac_child(a, v, c);
            if (u < 0) {
                u = ac_new_node(a, c, (int32_t)(j + 1));
                if (u < 0) { oracle_ac_free(a); return NULL; }
                a->nodes[u].next_sibling = a->nodes[v].first_child;
                a->nodes[v].first_child = u;
            }
            v = u;
        }
        /* append p to the node's id list, keeping ascending order */
        a->pid_next[p] = -1;
        if (a->nodes[v].pid_head < 0) {
            a->nodes[v].pid_head = (int32_t)p;
        } else {
            int32_t t = a->nodes[v].pid_head;
            while (a->pid_next[t] >= 0) t = a->pid_next[t];
            a->pid_next[t] = (int32_t)p;
        }
    }
    (void)pid_tail;

    /* 2. failure and output links, breadth first */
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)a->nnodes);
    if (!queue) { oracle_ac_free(a); return NULL; }
    int32_t qh = 0, qt = 0;
    for (int32_t u = a->nodes[0].first_child; u >= 0; u = a->nodes[u].next_sibling) {
        a->nodes[u].fail = 0;
        a->nodes[u].out = -1;
        queue[qt++] = u;
    }
    while (qh < qt) {
        int32_t v = queue[qh++];
        for (int32_t u = a->nodes[v].first_child; u >= 0; u = a->nodes[u].next_sibling) {
            uint8_t c = a->nodes[u].label;
            int32_t f = a->nodes[v].fail;
            int32_t g;
            while ((g = ac_child(a, f, c)) < 0 && f != 0) f = a->nodes[f].fail;
            a->nodes[u].fail = (g >= 0) ? g : 0;
            int32_t fu = a->nodes[u].fail;
            a->nodes[u].out = (a->nodes[fu].pid_head >= 0) ? fu : a->nodes[fu].out;
            queue[qt++] = u;
        }
    }
    free(queue);
    return a;
}

/* Builds the automaton for r patterns of length m (row-major in P). */
void *oracle_ac_build(const uint8_t *P, uint64_t r, uint64_t m)
{
    uint64_t *off = (uint64_t *)malloc(sizeof(uint64_t) * (r + 1));
    if (!off) return NULL;
    for (uint64_t p = 0; p <= r; p++) off[p] = p * m;
    void *a = oracle_ac_build_var(P, off, r);
    free(off);
    return a;
}

typedef struct {
    uint32_t *pos, *pid;
    uint64_t len, cap;
} occ_buf;

static int occ_push(occ_buf *b, uint32_t pos, uint32_t pid)
{
    if (b->len == b->cap) {
        uint64_t nc = b->cap ? b->cap * 2 : 256;
        uint32_t *np = (uint32_t *)realloc(b->pos, sizeof(uint32_t) * nc);
        if (!np) return -1;
        b->pos = np;
        uint32_t *nq = (uint32_t *)realloc(b->pid, sizeof(uint32_t) * nc);
        if (!nq) return -1;
        b->pid = nq;
        b->cap = nc;
    }
    b->pos[b->len] = pos;
    b->pid[b->len] = pid;
    b->len++;
    return 0;
}

/* Scans T[lo .. hi + m - 1) and keeps the occurrences starting in [lo, hi). */
static int ac_scan_range(const ac_automaton *a, const uint8_t *T, uint64_t n,
                         uint64_t lo, uint64_t hi, occ_buf *b)
{
    uint64_t end = hi + a->m - 1;
    if (end > n) end = n;
    int32_t v = 0;
    for (uint64_t j = lo; j < end; j++) {
        uint8_t c = T[j];
        int32_t g;
        while ((g = ac_child(a, v, c)) < 0 && v != 0) v = a->nodes[v].fail;
        v = (g >= 0) ? g : 0;
        /* report v and everything on its output chain */
        for (int32_t x = (a->nodes[v].pid_head >= 0) ? v : a->nodes[v].out; x >= 0;
             x = a->nodes[x].out) {
            uint64_t start = j + 1 - (uint64_t)a->nodes[x].depth;
            if (start < lo || start >= hi) continue;
            for (int32_t p = a->nodes[x].pid_head; p >= 0; p = a->pid_next[p])
                if (occ_push(b, (uint32_t)start, (uint32_t)p)) return -1;
        }
    }
    return 0;
}

typedef struct {
    const ac_automaton *a;
    const uint8_t *T;
    uint64_t n, lo, hi;
    occ_buf buf;
    int err;
} ac_job;

static void *ac_job_run(void *arg)
{
    ac_job *j = (ac_job *)arg;
    j->err = ac_scan_range(j->a, j->T, j->n, j->lo, j->hi, &j->buf);
    return NULL;
}

/* Returns the total number of occurrences (or -1 on allocation failure) and
 * writes at most `cap` of them, sorted by (position, pattern id) when all
 * patterns have one length (in order of their end position otherwise). */
int64_t oracle_ac_search(void *h, const uint8_t *T, uint64_t n, int threads,
                         uint32_t *out_pos, uint32_t *out_pid, uint64_t cap)
{
    const ac_automaton *a = (const ac_automaton *)h;
    if (!a || a->mmin == 0 || n < a->mmin) return 0;
    uint64_t starts = n - a->mmin + 1;
    if (threads < 1) threads = 1;
    if ((uint64_t)threads > starts) threads = (int)starts;
    ac_job *jobs = (ac_job *)calloc((size_t)threads, sizeof(ac_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tids) { free(jobs); free(tids); return -1; }
    for (int t = 0; t < threads; t++) {
        jobs[t].a = a;
        jobs[t].T = T;
        jobs[t].n = n;
        jobs[t].lo = starts * (uint64_t)t / (uint64_t)threads;
        jobs[t].hi = starts * (uint64_t)(t + 1) / (uint64_t)threads;
    }
    if (threads == 1) {
        ac_job_run(&jobs[0]);
    } else {
        for (int t = 0; t < threads; t++) pthread_create(&tids[t], NULL, ac_job_run, &jobs[t]);
        for (int t = 0; t < threads; t++) pthread_join(tids[t], NULL);
    }
    int64_t z = 0;
    int err = 0;
    for (int t = 0; t < threads; t++) {
        err |= jobs[t].err;
        for (uint64_t k = 0; k < jobs[t].buf.len; k++, z++) {
            if ((uint64_t)z < cap) {
                out_pos[z] = jobs[t].buf.pos[k];
                out_pid[z] = jobs[t].buf.pid[k];
            }
        }
        free(jobs[t].buf.pos);
        free(jobs[t].buf.pid);
    }
    free(jobs);
    free(tids);
    return err ? -1 : z;
}

/* Number of trie nodes (a sanity figure for the tests). */
int64_t oracle_ac_nodes(void *h)
{
    return h ? ((ac_automaton *)h)->nnodes : 0;
}
