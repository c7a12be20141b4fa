/* fq_cpu.c -- an all-cores OpenMP CPU baseline of the compressed-frontier BFS, for measurement.
 *
 * The same work as the GPU path, on the host's cores: a level-synchronous direction-optimising
 * BFS over CSR (top-down expansion of the sorted frontier queue, bottom-up sweep against the
 * frontier bitmap, switching by the rule top-down -> bottom-up when m_f * alpha > m_u and back
 * when n_f * beta < n; direction optimisation as in sec. 3.1 of the thesis) with every level's
 * frontier queue Q_d, frontier bitmap B_d and visited bitmap V_d encoded in the FQ / FB formats of
 * include/fqbfs.h (delta + binary packing in blocks of 128, sec. 5.1; packed only when smaller,
 * the losslessness requirement of sec. 5.1).  Every result is byte-identical to the plain oracle's; only the work is
 * spread over threads: the codec over 128-id blocks, the BFS over frontier vertices (top-down) or
 * 64-vertex words (bottom-up), the queue extraction over word ranges.
 *
 * It is neither the oracle (which stays plain and single-threaded) nor the product path (the CUDA
 * library); the benchmark times it beside them.  Little-endian hosts only (x86-64, Arm64).
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { CPU_OK = 0, CPU_EINVAL = 1, CPU_ENOMEM = 2, CPU_ENOSPC = 3, CPU_EUNSORTED = 5 };

#define BLK 128u
#define MAGIC_PACKED 0x31505146u /* "FQP1" */
#define MAGIC_RAW 0x31525146u    /* "FQR1" */
#define MAGIC_BITMAP 0x314D4246u /* "FBM1" */
#define FB_RAW 0u
#define FB_SET 1u
#define FB_CLEAR 2u

static inline uint32_t bitlen32(uint32_t x) { return x ? 32u - (uint32_t)__builtin_clz(x) : 0u; }
static inline uint64_t pad16(uint64_t b) { return (b + 15u) & ~(uint64_t)15u; }

/* ------------------------------------------------------------------ FQ */

/* Widths of the blocks of v[0..n) and their prefix (pre[nb] = sum); returns the stream size. */
static uint64_t fq_plan(const uint32_t *v, uint64_t n, uint8_t *w, uint64_t *pre, int *packed)
{
    const uint64_t nb = (n + BLK - 1u) / BLK;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < (int64_t)nb; k++) {
        const uint64_t i0 = (uint64_t)k * BLK, i1 = i0 + BLK < n ? i0 + BLK : n;
        uint32_t acc = 0;
        for (uint64_t i = i0 + 1; i < i1; i++) acc |= v[i] - v[i - 1] - 1u;
        w[k] = (uint8_t)bitlen32(acc);
    }
    pre[0] = 0;
    for (uint64_t k = 0; k < nb; k++) pre[k + 1] = pre[k] + w[k];
    const uint64_t ps = 16u + pad16(5u * nb) + 16u * pre[nb], rs = 16u + pad16(4u * n);
    *packed = n > 0 && ps < rs;
    return *packed ? ps : rs;
}

static void put32(uint8_t *p, uint32_t x) { memcpy(p, &x, 4); }

/* Write the FQ stream planned by fq_plan (out has room for size bytes). */
static void fq_write(const uint32_t *v, uint64_t n, const uint8_t *w, const uint64_t *pre, int packed, uint8_t *out,
                     uint64_t size)
{
    const uint64_t nb = (n + BLK - 1u) / BLK;
    memset(out, 0, size < 16u + pad16(5u * nb) ? size : 16u + pad16(5u * nb));
    if (!packed) {
        put32(out, MAGIC_RAW);
        put32(out + 4, (uint32_t)n);
        put32(out + 8, 0u);
        put32(out + 12, (uint32_t)n);
        memcpy(out + 16, v, 4u * n);
        memset(out + 16 + 4u * n, 0, size - 16u - 4u * n);
        return;
    }
    put32(out, MAGIC_PACKED);
    put32(out + 4, (uint32_t)n);
    put32(out + 8, (uint32_t)nb);
    put32(out + 12, (uint32_t)(4u * pre[nb]));
    const uint64_t payload = 16u + pad16(5u * nb);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < (int64_t)nb; k++) {
        put32(out + 16 + 4u * (uint64_t)k, v[(uint64_t)k * BLK]);
        out[16 + 4u * nb + (uint64_t)k] = w[k];
        const uint32_t b = w[k];
        uint32_t words[4 * 32];
        memset(words, 0, 16u * b);
        for (uint32_t j = 1; j < BLK && b; j++) {
            const uint64_t i = (uint64_t)k * BLK + j;
            if (i >= n) break;
            const uint32_t g = v[i] - v[i - 1] - 1u, pos = j * b, wd = pos >> 5, sh = pos & 31u;
            words[wd] |= g << sh;
            if (sh + b > 32u) words[wd + 1] |= g >> (32u - sh);
        }
        memcpy(out + payload + 16u * pre[k], words, 16u * b);
    }
}

/* FQ-encode the strictly increasing v[0..n) into out (capacity cap); *out_bytes = the size (also
 * on CPU_ENOSPC). */
int cpu_fq_encode(const uint32_t *v, uint64_t n, uint8_t *out, uint64_t cap, uint64_t *out_bytes)
{
    *out_bytes = 0;
    if (n > 0xFFFFFFFFull) return CPU_EINVAL;
    int bad = 0;
#pragma omp parallel for reduction(| : bad) schedule(static)
    for (int64_t i = 1; i < (int64_t)n; i++) bad |= v[i] <= v[i - 1];
    if (bad) return CPU_EUNSORTED;
    const uint64_t nb = (n + BLK - 1u) / BLK;
    uint8_t *w = malloc(nb ? nb : 1);
    uint64_t *pre = malloc(sizeof(uint64_t) * (nb + 1));
    if (!w || !pre) {
        free(w);
        free(pre);
        return CPU_ENOMEM;
    }
    int packed;
    const uint64_t size = fq_plan(v, n, w, pre, &packed);
    *out_bytes = size;
    int st = CPU_OK;
    if (size > cap) st = CPU_ENOSPC;
    else fq_write(v, n, w, pre, packed, out, size);
    free(w);
    free(pre);
    return st;
}

/* ------------------------------------------------------------------ bitmaps */

static inline uint64_t masked_word(const uint64_t *words, uint64_t i, uint64_t nbits)
{
    const uint64_t nw = (nbits + 63u) / 64u;
    uint64_t x = words[i];
    if (i == nw - 1 && (nbits & 63u)) x &= (1ull << (nbits & 63u)) - 1ull;
    return x;
}

/* Sorted positions of the set bits (invert = 0) or of the clear bits below nbits (invert = 1) into
 * pos; returns their count.  Parallel over word ranges (counts, prefix, fill). */
static uint64_t positions(const uint64_t *words, uint64_t nbits, int invert, uint32_t *pos)
{
    const uint64_t nw = (nbits + 63u) / 64u;
    const int nt = omp_get_max_threads();
    uint64_t *cnt = calloc((size_t)nt + 1, sizeof(uint64_t));
    int used = 1;
#pragma omp parallel num_threads(nt)
    {
        const int t = omp_get_thread_num(), T = omp_get_num_threads();
        if (t == 0) used = T;
        const uint64_t w0 = nw * (uint64_t)t / (uint64_t)T, w1 = nw * (uint64_t)(t + 1) / (uint64_t)T;
        uint64_t c = 0;
        for (uint64_t i = w0; i < w1; i++) {
            uint64_t x = masked_word(words, i, nbits);
            if (invert) {
                x = ~x;
                if (i == nw - 1 && (nbits & 63u)) x &= (1ull << (nbits & 63u)) - 1ull;
            }
            c += (uint64_t)__builtin_popcountll(x);
        }
        cnt[t + 1] = c;
#pragma omp barrier
#pragma omp single
        for (int i = 0; i < T; i++) cnt[i + 1] += cnt[i];
        uint64_t o = cnt[t];
        for (uint64_t i = w0; i < w1; i++) {
            uint64_t x = masked_word(words, i, nbits);
            if (invert) {
                x = ~x;
                if (i == nw - 1 && (nbits & 63u)) x &= (1ull << (nbits & 63u)) - 1ull;
            }
            while (x) {
                pos[o++] = (uint32_t)(64u * i + (uint64_t)__builtin_ctzll(x));
                x &= x - 1u;
            }
        }
    }
    const uint64_t total = cnt[used];
    free(cnt);
    return total;
}

/* FB-encode the bitmap (nbits <= 2^32) into out (capacity cap); *out_bytes = the size. */
int cpu_fb_encode(const uint64_t *words, uint64_t nbits, uint8_t *out, uint64_t cap, uint64_t *out_bytes)
{
    *out_bytes = 0;
    if (nbits > (1ull << 32)) return CPU_EINVAL;
    const uint64_t nw = (nbits + 63u) / 64u;
    uint64_t P = 0;
#pragma omp parallel for reduction(+ : P) schedule(static)
    for (int64_t i = 0; i < (int64_t)nw; i++) P += (uint64_t)__builtin_popcountll(masked_word(words, (uint64_t)i, nbits));
    const uint32_t mode = 2u * P <= nbits ? FB_SET : FB_CLEAR;
    const uint64_t c = mode == FB_SET ? P : nbits - P;
    const uint64_t raw = 16u + pad16(8u * nw);
    uint32_t *pos = malloc(sizeof(uint32_t) * (c ? c : 1));
    const uint64_t nb = (c + BLK - 1u) / BLK;
    uint8_t *w = malloc(nb ? nb : 1);
    uint64_t *pre = malloc(sizeof(uint64_t) * (nb + 1));
    if (!pos || !w || !pre) {
        free(pos);
        free(w);
        free(pre);
        return CPU_ENOMEM;
    }
    positions(words, nbits, mode == FB_CLEAR, pos);
    int packed;
    const uint64_t inner = fq_plan(pos, c, w, pre, &packed);
    const int use_raw = 16u + inner >= raw;
    const uint64_t size = use_raw ? raw : 16u + inner;
    *out_bytes = size;
    int st = CPU_OK;
    if (size > cap) {
        st = CPU_ENOSPC;
    } else {
        put32(out, MAGIC_BITMAP);
        put32(out + 4, use_raw ? FB_RAW : mode);
        memcpy(out + 8, &nbits, 8);
        if (use_raw) {
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < (int64_t)nw; i++) {
                const uint64_t x = masked_word(words, (uint64_t)i, nbits);
                memcpy(out + 16 + 8u * (uint64_t)i, &x, 8);
            }
            memset(out + 16 + 8u * nw, 0, raw - 16u - 8u * nw);
        } else {
            fq_write(pos, c, w, pre, packed, out + 16, inner);
        }
    }
    free(pos);
    free(w);
    free(pre);
    return st;
}

/* ------------------------------------------------------------------ BFS */

/* BFS from root.  depth[n] (-1 unreached), parent[n] (parent[root] = root, unreached 2^32 - 1).
 * Every level's Q_d, B_d and (visited_stream) V_d are encoded; their total size lands in
 * *stream_bytes.  With log != NULL the streams are also written there back to back (Q, B, V per
 * level; log_sizes[3 d .. 3 d + 2] their sizes; at most max_levels levels, CPU_ENOSPC past
 * log_cap).  *levels = levels with a non-empty frontier; *reached_edges = undirected edges inside
 * the reached component. */
int cpu_bfs(uint64_t n, const int64_t *off, const uint32_t *cols, uint32_t root, uint32_t alpha, uint32_t beta,
            int visited_stream, int32_t *depth, uint32_t *parent, uint64_t *stream_bytes, uint32_t *levels,
            uint64_t *reached_edges, uint8_t *log, uint64_t log_cap, uint64_t *log_sizes, uint32_t max_levels)
{
    if (n == 0 || n > 0xFFFFFFFFull || root >= n) return CPU_EINVAL;
    const uint64_t nw = (n + 63u) / 64u;
    uint64_t *front = calloc(nw, 8), *next = calloc(nw, 8), *vis = calloc(nw, 8);
    uint32_t *q = malloc(4u * n), *q2 = malloc(4u * n);
    const uint64_t bound = 16u + pad16(8u * nw) + 16u + pad16(4u * n);  /* any FQ or FB stream */
    uint8_t *buf = malloc(bound);
    if (!front || !next || !vis || !q || !q2 || !buf) {
        free(front); free(next); free(vis); free(q); free(q2); free(buf);
        return CPU_ENOMEM;
    }
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < (int64_t)n; v++) {
        depth[v] = -1;
        parent[v] = 0xFFFFFFFFu;
    }
    uint64_t total_deg = (uint64_t)off[n] - (uint64_t)off[0];
    depth[root] = 0;
    parent[root] = root;
    q[0] = root;
    uint64_t nf = 1, visited_deg = 0, bytes = 0, logged = 0;
    front[root >> 6] |= 1ull << (root & 63u);
    vis[root >> 6] |= 1ull << (root & 63u);
    int td = 1, st = CPU_OK;
    uint32_t d = 0;
    while (nf > 0) {
        uint64_t mf = 0;
#pragma omp parallel for reduction(+ : mf) schedule(static)
        for (int64_t i = 0; i < (int64_t)nf; i++) mf += (uint64_t)(off[q[i] + 1] - off[q[i]]);
        visited_deg += mf;
        const uint64_t mu = total_deg - visited_deg;
        if (td && mf * alpha > mu) td = 0;
        else if (!td && nf * beta < n) td = 1;
        /* this level's streams */
        uint64_t sz[3] = {0, 0, 0};
        cpu_fq_encode(q, nf, buf, bound, &sz[0]);
        if (log && d < max_levels && logged + sz[0] <= log_cap) memcpy(log + logged, buf, sz[0]);
        uint64_t l0 = logged + sz[0];
        cpu_fb_encode(front, n, buf, bound, &sz[1]);
        if (log && d < max_levels && l0 + sz[1] <= log_cap) memcpy(log + l0, buf, sz[1]);
        uint64_t l1 = l0 + sz[1];
        if (visited_stream) {
            cpu_fb_encode(vis, n, buf, bound, &sz[2]);
            if (log && d < max_levels && l1 + sz[2] <= log_cap) memcpy(log + l1, buf, sz[2]);
        }
        bytes += sz[0] + sz[1] + sz[2];
        if (log) {
            if (d >= max_levels || l1 + sz[2] > log_cap) st = CPU_ENOSPC;
            else {
                log_sizes[3u * d] = sz[0];
                log_sizes[3u * d + 1] = sz[1];
                log_sizes[3u * d + 2] = sz[2];
            }
            logged = l1 + sz[2];
        }
        /* expand into next */
        memset(next, 0, 8u * nw);
        const int32_t nd = (int32_t)d + 1;
        if (td) {
#pragma omp parallel for schedule(dynamic, 64)
            for (int64_t i = 0; i < (int64_t)nf; i++) {
                const uint32_t v = q[i];
                for (int64_t e = off[v]; e < off[v + 1]; e++) {
                    const uint32_t w = cols[e];
                    const uint64_t bit = 1ull << (w & 63u);
                    if (vis[w >> 6] & bit) continue;
                    if (__atomic_load_n(&next[w >> 6], __ATOMIC_RELAXED) & bit) continue;
                    if (!(__atomic_fetch_or(&next[w >> 6], bit, __ATOMIC_RELAXED) & bit)) {
                        depth[w] = nd;
                        parent[w] = v;
                    }
                }
            }
        } else {
#pragma omp parallel for schedule(dynamic, 256)
            for (int64_t wi = 0; wi < (int64_t)nw; wi++) {
                uint64_t un = ~vis[wi], found = 0;
                if (wi == (int64_t)nw - 1 && (n & 63u)) un &= (1ull << (n & 63u)) - 1ull;
                while (un) {
                    const uint32_t b = (uint32_t)__builtin_ctzll(un);
                    un &= un - 1u;
                    const uint64_t w = 64u * (uint64_t)wi + b;
                    for (int64_t e = off[w]; e < off[w + 1]; e++) {
                        const uint32_t u = cols[e];
                        if (front[u >> 6] & (1ull << (u & 63u))) {
                            depth[w] = nd;
                            parent[w] = u;
                            found |= 1ull << b;
                            break;
                        }
                    }
                }
                next[wi] = found;
            }
        }
        /* next frontier: sorted queue, visited |= next */
        nf = positions(next, n, 0, q2);
        uint32_t *t = q; q = q2; q2 = t;
        uint64_t *tb = front; front = next; next = tb;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < (int64_t)nw; i++) vis[i] |= front[i];
        d++;
    }
    uint64_t re = 0;
#pragma omp parallel for reduction(+ : re) schedule(static)
    for (int64_t v = 0; v < (int64_t)n; v++)
        if (depth[v] >= 0) re += (uint64_t)(off[v + 1] - off[v]);
    *reached_edges = re / 2u;
    *levels = d;
    *stream_bytes = bytes;
    free(front); free(next); free(vis); free(q); free(q2); free(buf);
    return st;
}

int cpu_threads(void) { return omp_get_max_threads(); }

void cpu_set_threads(int t) { omp_set_num_threads(t > 0 ? t : 1); }
