/*
 * fq_oracle.c -- plain, slow, single-threaded CPU oracle for the compressed-frontier BFS.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call this file:
 * only the test suite, the package smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header, table or constant generator with the CUDA library; it restates
 * the method from the thesis "Optimizing Communication by Compression for Multi-GPU Scalable
 * Breadth-First Searches" (arXiv 1704.00513) in the most direct form available.
 *
 * Contents (each function cites the passage it follows):
 *   orc_bfs            textbook FIFO-queue BFS -> hop depth and a BFS tree
 *                      (Algorithm 2, sec. 4.1.2)
 *   orc_validate       BFS-tree checks (the "5 rules" of Graph500 validation, Algorithm 1;
 *                      the rules are not listed in the thesis, our reading)
 *   orc_fq_encode/decode  delta + frame-of-reference binary packing in blocks of 128
 *                      (binary packing and delta coding, sec. 5.1; S4-BP128 in sec. 5.3;
 *                      width formula Eq. 6/7), written bit by bit
 *   orc_px_encode/decode  binary packing with patched exceptions (patched coding, sec. 5.1,
 *                      Eq. 8-9; the PFOR family in sec. 5.3): per block
 *                      the width b that minimises the block's bytes, gaps >= 2^b stored apart
 *   orc_fr_encode/decode  frame of reference without differencing (Eq. 5-6 as printed: per block
 *                      the minimum as base, width = bit length of max - min) for unsorted values
 *   orc_fb_encode/decode  frontier/visited bitmap codec: positions of the minority bit value,
 *                      coded with the queue codec, or the raw words (bitmap frontiers and the
 *                      popcount-indexed sparse vector, sec. 3.1; lossless requirement, sec. 5.1)
 *   orc_bu_examined    edges a bottom-up sweep examines at one level (direction optimisation,
 *                      sec. 3.1)
 *
 * Integers only; no floating point anywhere.  Every routine is O(size) or O(size * 32) with
 * no blocking, fusion or reordering beyond the definitions.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* status codes of the oracle (same meanings as the library's, defined independently) */
enum {
    ORC_OK = 0,
    ORC_EINVAL = 1,
    ORC_ENOMEM = 2,
    ORC_ENOSPC = 3,
    ORC_ECORRUPT = 4,
    ORC_EUNSORTED = 5
};

/* stream magics: the ASCII bytes 'F','Q','P','1' etc. read as a little-endian u32 */
#define ORC_MAGIC_PACKED ((uint32_t)'F' | ((uint32_t)'Q' << 8) | ((uint32_t)'P' << 16) | ((uint32_t)'1' << 24))
#define ORC_MAGIC_RAW    ((uint32_t)'F' | ((uint32_t)'Q' << 8) | ((uint32_t)'R' << 16) | ((uint32_t)'1' << 24))
#define ORC_MAGIC_BITMAP ((uint32_t)'F' | ((uint32_t)'B' << 8) | ((uint32_t)'M' << 16) | ((uint32_t)'1' << 24))
#define ORC_MAGIC_PATCHED ((uint32_t)'F' | ((uint32_t)'Q' << 8) | ((uint32_t)'X' << 16) | ((uint32_t)'1' << 24))
#define ORC_MAGIC_FOR ((uint32_t)'F' | ((uint32_t)'R' << 8) | ((uint32_t)'P' << 16) | ((uint32_t)'1' << 24))
#define ORC_MAGIC_FOR_RAW ((uint32_t)'F' | ((uint32_t)'R' << 8) | ((uint32_t)'R' << 16) | ((uint32_t)'1' << 24))

#define ORC_BLOCK 128u /* B, the block length of binary packing (sec. 5.1, S4-BP128 in sec. 5.3) */

enum { ORC_FB_RAW = 0, ORC_FB_SET = 1, ORC_FB_CLEAR = 2 };

/* ------------------------------------------------------------------ small helpers */

/* number of bits needed to write x in binary; bitlen(0) = 0.  This is Eq. 6 read as a
 * ceiling: ceil(log2(x + 1)) -- e.g. the range 2000..2127 needs bitlen(127) = 7 (Eq. 7). */
uint32_t orc_bitlen(uint64_t x)
{
    uint32_t bits = 0;
    while (x != 0) {
        x >>= 1;
        bits++;
    }
    return bits;
}

static uint64_t pad16(uint64_t bytes) { return (bytes + 15u) / 16u * 16u; }

static void put_u32(uint8_t *p, uint32_t x)
{
    p[0] = (uint8_t)(x & 0xFFu);
    p[1] = (uint8_t)((x >> 8) & 0xFFu);
    p[2] = (uint8_t)((x >> 16) & 0xFFu);
    p[3] = (uint8_t)((x >> 24) & 0xFFu);
}

static uint32_t get_u32(const uint8_t *p)
{
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

static void put_u64(uint8_t *p, uint64_t x)
{
    put_u32(p, (uint32_t)(x & 0xFFFFFFFFu));
    put_u32(p + 4, (uint32_t)(x >> 32));
}

static uint64_t get_u64(const uint8_t *p) { return (uint64_t)get_u32(p) | ((uint64_t)get_u32(p + 4) << 32); }

/* bit t of a byte buffer, least significant bit of byte 0 first.  A little-endian u32 word w
 * holds bits 32w .. 32w+31 of this numbering, so "bit t is bit (t mod 32) of word t/32". */
static void set_bit(uint8_t *buf, uint64_t t) { buf[t / 8u] = (uint8_t)(buf[t / 8u] | (1u << (t % 8u))); }
static uint32_t get_bit(const uint8_t *buf, uint64_t t) { return (uint32_t)((buf[t / 8u] >> (t % 8u)) & 1u); }

/* ------------------------------------------------------------------ queue codec "FQ"
 *
 * Input: a strictly increasing sequence v[0..n) of uint32 (a frontier queue is a sorted set,
 * sec. 4.1.4).  Blocks of B = 128 slots.  In block k, slot 0 holds 0 (the block's first value is
 * stored whole as base_k, the frame of reference, Eq. 5), slot j >= 1 holds the d-gap
 * v[128k+j] - v[128k+j-1] - 1 (delta coding, sec. 5.1; the "- 1" uses uniqueness), and slots
 * past n hold 0.  The block width b_k is the bit length of its largest slot (Eq. 6), so every
 * slot fits in b_k bits.  Slot j occupies bits [j*b_k, (j+1)*b_k) of the block's bit string.
 *
 * Packed stream: header u32[4] = {magic "FQP1", n, nb, payload_words}, u32 base[nb],
 * u8 b[nb], zeros up to a 16-byte boundary, then the nb bit strings (block k is 4*b_k u32
 * words).  Raw stream: {magic "FQR1", n, 0, n}, u32 v[n], zeros up to 16 bytes.  The packed
 * form is used only when strictly smaller (the encoded data must be smaller than the input,
 * the losslessness requirement of sec. 5.1; compression threshold, sec. 5.4.3), so ties and n = 0 are raw.
 */

uint64_t orc_fq_raw_size(uint64_t n) { return 16u + pad16(4u * n); }

int orc_fq_encode(const uint32_t *v, uint64_t n, uint8_t *out, uint64_t cap, uint64_t *out_bytes)
{
    uint64_t nb, k, j, t, i, sum_b = 0, size, packed_size, raw_size, payload_start, bit0;
    uint8_t *b;
    int packed;

    *out_bytes = 0;
    if (n > 0xFFFFFFFFu)
        return ORC_EINVAL;
    for (i = 1; i < n; i++)
        if (v[i] <= v[i - 1])
            return ORC_EUNSORTED;

    nb = (n + ORC_BLOCK - 1u) / ORC_BLOCK;
    b = (uint8_t *)calloc(nb ? nb : 1u, 1);
    if (!b)
        return ORC_ENOMEM;
    for (k = 0; k < nb; k++) {
        uint64_t max_gap = 0;
        for (j = 1; j < ORC_BLOCK; j++) {
            i = k * ORC_BLOCK + j;
            if (i < n) {
                uint64_t gap = (uint64_t)v[i] - (uint64_t)v[i - 1] - 1u;
                if (gap > max_gap)
                    max_gap = gap;
            }
        }
        b[k] = (uint8_t)orc_bitlen(max_gap);
        sum_b += b[k];
    }

    packed_size = 16u + pad16(5u * nb) + 16u * sum_b;
    raw_size = orc_fq_raw_size(n);
    packed = (n > 0) && (packed_size < raw_size);
    size = packed ? packed_size : raw_size;
    *out_bytes = size;
    if (size > cap) {
        free(b);
        return ORC_ENOSPC;
    }
    memset(out, 0, size);

    if (!packed) {
        put_u32(out + 0, ORC_MAGIC_RAW);
        put_u32(out + 4, (uint32_t)n);
        put_u32(out + 8, 0u);
        put_u32(out + 12, (uint32_t)n);
        for (i = 0; i < n; i++)
            put_u32(out + 16u + 4u * i, v[i]);
        free(b);
        return ORC_OK;
    }

    put_u32(out + 0, ORC_MAGIC_PACKED);
    put_u32(out + 4, (uint32_t)n);
    put_u32(out + 8, (uint32_t)nb);
    put_u32(out + 12, (uint32_t)(4u * sum_b));
    for (k = 0; k < nb; k++) {
        put_u32(out + 16u + 4u * k, v[k * ORC_BLOCK]);
        out[16u + 4u * nb + k] = b[k];
    }
    payload_start = 16u + pad16(5u * nb);
    bit0 = 8u * payload_start; /* first bit of block 0 */
    for (k = 0; k < nb; k++) {
        for (j = 0; j < ORC_BLOCK; j++) {
            uint64_t gap = 0;
            i = k * ORC_BLOCK + j;
            if (j > 0 && i < n)
                gap = (uint64_t)v[i] - (uint64_t)v[i - 1] - 1u;
            for (t = 0; t < b[k]; t++)
                if ((gap >> t) & 1u)
                    set_bit(out, bit0 + j * b[k] + t);
        }
        bit0 += 128u * b[k]; /* the block's 4*b_k words */
    }
    free(b);
    return ORC_OK;
}

/* Inverse of orc_fq_encode.  Rejects (ORC_ECORRUPT) any stream whose header, widths, sizes,
 * padding or decoded values are inconsistent: unknown magic, nb != ceil(n/128), a width > 32,
 * payload_words != 4*sum(b), in_bytes != the layout's size, nonzero pad bits or bytes, a
 * nonzero slot 0 or padding slot, or values that are not strictly increasing / overflow u32.
 * n > cap gives ORC_ENOSPC with *n_out = n. */
int orc_fq_decode(const uint8_t *in, uint64_t in_bytes, uint32_t *out, uint64_t cap, uint64_t *n_out)
{
    uint32_t magic;
    uint64_t n, nb, words, k, j, t, i, sum_b = 0, payload_start, bit0;

    *n_out = 0;
    if (in_bytes < 16u)
        return ORC_ECORRUPT;
    magic = get_u32(in);
    n = get_u32(in + 4);
    nb = get_u32(in + 8);
    words = get_u32(in + 12);

    if (magic == ORC_MAGIC_RAW) {
        if (nb != 0u || words != n || in_bytes != orc_fq_raw_size(n))
            return ORC_ECORRUPT;
        for (i = 16u + 4u * n; i < in_bytes; i++)
            if (in[i] != 0u)
                return ORC_ECORRUPT;
        for (i = 1; i < n; i++)
            if (get_u32(in + 16u + 4u * i) <= get_u32(in + 16u + 4u * (i - 1u)))
                return ORC_ECORRUPT;
        *n_out = n;
        if (n > cap)
            return ORC_ENOSPC;
        for (i = 0; i < n; i++)
            out[i] = get_u32(in + 16u + 4u * i);
        return ORC_OK;
    }
    if (magic != ORC_MAGIC_PACKED)
        return ORC_ECORRUPT;
    if (nb != (n + ORC_BLOCK - 1u) / ORC_BLOCK)
        return ORC_ECORRUPT;
    if (in_bytes < 16u + pad16(5u * nb))
        return ORC_ECORRUPT;
    for (k = 0; k < nb; k++) {
        uint32_t bk = in[16u + 4u * nb + k];
        if (bk > 32u)
            return ORC_ECORRUPT;
        sum_b += bk;
    }
    payload_start = 16u + pad16(5u * nb);
    if (words != 4u * sum_b || in_bytes != payload_start + 16u * sum_b)
        return ORC_ECORRUPT;
    for (i = 16u + 5u * nb; i < payload_start; i++)
        if (in[i] != 0u)
            return ORC_ECORRUPT;
    *n_out = n;
    if (n > cap)
        return ORC_ENOSPC;

    bit0 = 8u * payload_start;
    for (k = 0; k < nb; k++) {
        uint32_t bk = in[16u + 4u * nb + k];
        uint64_t value = get_u32(in + 16u + 4u * k); /* base_k */
        for (j = 0; j < ORC_BLOCK; j++) {
            uint64_t gap = 0;
            for (t = 0; t < bk; t++)
                gap |= (uint64_t)get_bit(in, bit0 + j * bk + t) << t;
            i = k * ORC_BLOCK + j;
            if (j == 0 || i >= n) {
                if (gap != 0u)
                    return ORC_ECORRUPT;
                if (j == 0) {
                    if (k > 0 && value <= out[i - 1u])
                        return ORC_ECORRUPT;
                    out[i] = (uint32_t)value;
                }
                continue;
            }
            value = value + gap + 1u;
            if (value > 0xFFFFFFFFu)
                return ORC_ECORRUPT;
            out[i] = (uint32_t)value;
        }
        bit0 += 128u * bk;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ patched codec "PX"
 *
 * Binary packing with exceptions (patched coding, sec. 5.1: a value that does
 * not fit in the block's b bits -- a gap >= 2^b, Eq. 8-9 -- is stored apart; PFOR family,
 * sec. 5.3).  Same gaps, blocks and raw fallback as FQ.  Per block k the width b_k is the b in
 * 0..32 that minimises the block's bytes 16*b + 5*e_b, e_b = number of gaps >= 2^b (each
 * exception costs a u8 slot position and a u32 high part); ties go to the larger b.  Layout
 * (all u32 little-endian, every section starting on a 16-byte boundary):
 *   header 32 B : "FQX1", n, nb, payload_words = 4*sum(b), E = sum(e), 0, 0, 0
 *   u32 base[nb], u8 b[nb], u8 e[nb], zero pad to 16
 *   payload     : per block 4*b_k words, slot j's low b_k gap bits at [j*b_k, (j+1)*b_k)
 *   u8 pos[E]   : per block in order, its exception slots (1..127, increasing), zero pad to 16
 *   u32 high[E] : gap >> b_k of each exception, zero pad to 16
 * The packed form is used only if strictly smaller than the raw FQ form (which it then is).
 */

uint64_t orc_px_size(uint64_t nb, uint64_t sum_b, uint64_t e_total)
{
    return 32u + pad16(6u * nb) + 16u * sum_b + pad16(e_total) + pad16(4u * e_total);
}

/* the width and exception count of one block of gaps g[0..cnt) (slot 0 included, always 0) */
static void px_choose(const uint64_t *g, uint64_t cnt, uint32_t *b_out, uint32_t *e_out)
{
    uint32_t b, best_b = 32;
    uint64_t best_cost = 16u * 32u, j;
    for (b = 0; b <= 32u; b++) {
        uint64_t e = 0, cost;
        for (j = 0; j < cnt; j++)
            if (b < 32u && (g[j] >> b) != 0u)
                e++;
        cost = 16u * b + 5u * e;
        if (cost <= best_cost) { /* <=: a tie moves to the larger b */
            best_cost = cost;
            best_b = b;
        }
    }
    *b_out = best_b;
    *e_out = 0;
    for (j = 0; j < cnt; j++)
        if (best_b < 32u && (g[j] >> best_b) != 0u)
            (*e_out)++;
}

int orc_px_encode(const uint32_t *v, uint64_t n, uint8_t *out, uint64_t cap, uint64_t *out_bytes)
{
    uint64_t nb, k, j, t, i, sum_b = 0, e_total = 0, size, packed_size, raw_size, payload, bit0, xpos, xhigh, x;
    uint8_t *b, *e;
    uint64_t g[ORC_BLOCK];
    int packed;

    *out_bytes = 0;
    if (n > 0xFFFFFFFFu)
        return ORC_EINVAL;
    for (i = 1; i < n; i++)
        if (v[i] <= v[i - 1])
            return ORC_EUNSORTED;
    nb = (n + ORC_BLOCK - 1u) / ORC_BLOCK;
    b = (uint8_t *)calloc(nb ? nb : 1u, 1);
    e = (uint8_t *)calloc(nb ? nb : 1u, 1);
    if (!b || !e) {
        free(b);
        free(e);
        return ORC_ENOMEM;
    }
    for (k = 0; k < nb; k++) {
        uint32_t bk, ek;
        uint64_t cnt = 0;
        for (j = 0; j < ORC_BLOCK; j++) {
            i = k * ORC_BLOCK + j;
            if (i >= n)
                break;
            g[cnt++] = j == 0 ? 0u : (uint64_t)v[i] - (uint64_t)v[i - 1] - 1u;
        }
        px_choose(g, cnt, &bk, &ek);
        b[k] = (uint8_t)bk;
        e[k] = (uint8_t)ek;
        sum_b += bk;
        e_total += ek;
    }
    packed_size = orc_px_size(nb, sum_b, e_total);
    raw_size = orc_fq_raw_size(n);
    packed = (n > 0) && (packed_size < raw_size);
    size = packed ? packed_size : raw_size;
    *out_bytes = size;
    if (size > cap) {
        free(b);
        free(e);
        return ORC_ENOSPC;
    }
    memset(out, 0, size);
    if (!packed) { /* the raw FQ form */
        put_u32(out + 0, ORC_MAGIC_RAW);
        put_u32(out + 4, (uint32_t)n);
        put_u32(out + 8, 0u);
        put_u32(out + 12, (uint32_t)n);
        for (i = 0; i < n; i++)
            put_u32(out + 16u + 4u * i, v[i]);
        free(b);
        free(e);
        return ORC_OK;
    }
    put_u32(out + 0, ORC_MAGIC_PATCHED);
    put_u32(out + 4, (uint32_t)n);
    put_u32(out + 8, (uint32_t)nb);
    put_u32(out + 12, (uint32_t)(4u * sum_b));
    put_u32(out + 16, (uint32_t)e_total);
    for (k = 0; k < nb; k++) {
        put_u32(out + 32u + 4u * k, v[k * ORC_BLOCK]);
        out[32u + 4u * nb + k] = b[k];
        out[32u + 5u * nb + k] = e[k];
    }
    payload = 32u + pad16(6u * nb);
    xpos = payload + 16u * sum_b;
    xhigh = xpos + pad16(e_total);
    bit0 = 8u * payload;
    x = 0; /* exceptions written so far */
    for (k = 0; k < nb; k++) {
        for (j = 0; j < ORC_BLOCK; j++) {
            uint64_t gap = 0;
            i = k * ORC_BLOCK + j;
            if (j > 0 && i < n)
                gap = (uint64_t)v[i] - (uint64_t)v[i - 1] - 1u;
            for (t = 0; t < b[k]; t++)
                if ((gap >> t) & 1u)
                    set_bit(out, bit0 + j * b[k] + t);
            if (b[k] < 32u && (gap >> b[k]) != 0u) { /* an exception: slot and high part */
                out[xpos + x] = (uint8_t)j;
                put_u32(out + xhigh + 4u * x, (uint32_t)(gap >> b[k]));
                x++;
            }
        }
        bit0 += 128u * b[k];
    }
    free(b);
    free(e);
    return ORC_OK;
}

/* Inverse of orc_px_encode (and of the raw FQ form).  Rejects (ORC_ECORRUPT): unknown magic,
 * nb != ceil(n/128), nonzero reserved header words, a width > 32, more than 127 exceptions in a
 * block or any with width 32, payload_words != 4*sum(b), E != sum(e), in_bytes != the layout's
 * size, nonzero pads, exception slots that are not increasing within 1..127 or that fall past
 * n, a zero high part or one that does not fit above the width, a nonzero slot 0 or padding
 * slot, and values that overflow u32.  n > cap gives ORC_ENOSPC with *n_out = n. */
int orc_px_decode(const uint8_t *in, uint64_t in_bytes, uint32_t *out, uint64_t cap, uint64_t *n_out)
{
    uint64_t n, nb, words, e_total, k, j, t, i, sum_b = 0, sum_e = 0, payload, xpos, xhigh, bit0, x;
    uint64_t g[ORC_BLOCK];

    *n_out = 0;
    if (in_bytes < 16u)
        return ORC_ECORRUPT;
    if (get_u32(in) == ORC_MAGIC_RAW)
        return orc_fq_decode(in, in_bytes, out, cap, n_out);
    if (get_u32(in) != ORC_MAGIC_PATCHED || in_bytes < 32u)
        return ORC_ECORRUPT;
    n = get_u32(in + 4);
    nb = get_u32(in + 8);
    words = get_u32(in + 12);
    e_total = get_u32(in + 16);
    if (get_u32(in + 20) || get_u32(in + 24) || get_u32(in + 28))
        return ORC_ECORRUPT;
    if (nb != (n + ORC_BLOCK - 1u) / ORC_BLOCK || in_bytes < 32u + pad16(6u * nb))
        return ORC_ECORRUPT;
    for (k = 0; k < nb; k++) {
        uint32_t bk = in[32u + 4u * nb + k], ek = in[32u + 5u * nb + k];
        if (bk > 32u || ek > 127u || (bk == 32u && ek != 0u))
            return ORC_ECORRUPT;
        sum_b += bk;
        sum_e += ek;
    }
    payload = 32u + pad16(6u * nb);
    if (words != 4u * sum_b || e_total != sum_e || in_bytes != orc_px_size(nb, sum_b, sum_e))
        return ORC_ECORRUPT;
    xpos = payload + 16u * sum_b;
    xhigh = xpos + pad16(sum_e);
    for (i = 32u + 6u * nb; i < payload; i++)
        if (in[i] != 0u)
            return ORC_ECORRUPT;
    for (i = xpos + sum_e; i < xhigh; i++)
        if (in[i] != 0u)
            return ORC_ECORRUPT;
    for (i = xhigh + 4u * sum_e; i < in_bytes; i++)
        if (in[i] != 0u)
            return ORC_ECORRUPT;
    *n_out = n;
    if (n > cap)
        return ORC_ENOSPC;

    bit0 = 8u * payload;
    x = 0;
    for (k = 0; k < nb; k++) {
        uint32_t bk = in[32u + 4u * nb + k], ek = in[32u + 5u * nb + k], q;
        uint64_t value = get_u32(in + 32u + 4u * k), last = 0;
        for (j = 0; j < ORC_BLOCK; j++) { /* the low bits of every slot */
            g[j] = 0;
            for (t = 0; t < bk; t++)
                g[j] |= (uint64_t)get_bit(in, bit0 + j * bk + t) << t;
        }
        for (q = 0; q < ek; q++, x++) { /* patch the exceptions */
            uint64_t slot = in[xpos + x], high = get_u32(in + xhigh + 4u * x);
            if (slot == 0u || slot <= last || k * ORC_BLOCK + slot >= n)
                return ORC_ECORRUPT;
            if (high == 0u || (high >> (32u - bk)) != 0u)
                return ORC_ECORRUPT;
            last = slot;
            g[slot] |= high << bk;
        }
        for (j = 0; j < ORC_BLOCK; j++) {
            i = k * ORC_BLOCK + j;
            if (j == 0 || i >= n) {
                if (g[j] != 0u)
                    return ORC_ECORRUPT;
                if (j == 0) {
                    if (k > 0 && value <= out[i - 1u])
                        return ORC_ECORRUPT;
                    out[i] = (uint32_t)value;
                }
                continue;
            }
            value = value + g[j] + 1u;
            if (value > 0xFFFFFFFFu)
                return ORC_ECORRUPT;
            out[i] = (uint32_t)value;
        }
        bit0 += 128u * bk;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ frame of reference "FR"
 *
 * Unsorted u32 values in blocks of 128 (Eq. 5: every value of a block is stored as its offset from
 * the block's minimum; Eq. 6: the block's width is the bit length of max - min).  Layout:
 *   packed {u32 "FRP1", n, nb, payload_words = 4*sum(b)}, u32 min[nb], u8 b[nb], zero pad to 16,
 *          per block 4*b_k words, slot j = v[128k+j] - min_k at bits [j*b_k, (j+1)*b_k), slots
 *          past n are 0;
 *   raw    {u32 "FRR1", n, 0, n}, u32 v[n], zero pad to 16.
 * The packed form is written only when strictly smaller than the raw one.
 */

uint64_t orc_fr_size(uint64_t nb, uint64_t sum_b) { return 16u + pad16(5u * nb) + 16u * sum_b; }

int orc_fr_encode(const uint32_t *v, uint64_t n, uint8_t *out, uint64_t cap, uint64_t *out_bytes)
{
    uint64_t nb, k, j, t, i, sum_b = 0, size, packed_size, raw_size, bit0;
    uint8_t *b;
    uint32_t *mn;
    int packed;

    *out_bytes = 0;
    if (n > 0xFFFFFFFFu)
        return ORC_EINVAL;
    nb = (n + ORC_BLOCK - 1u) / ORC_BLOCK;
    b = (uint8_t *)calloc(nb ? nb : 1u, 1);
    mn = (uint32_t *)calloc(nb ? nb : 1u, sizeof(uint32_t));
    if (!b || !mn) {
        free(b);
        free(mn);
        return ORC_ENOMEM;
    }
    for (k = 0; k < nb; k++) {
        uint32_t lo = 0xFFFFFFFFu, hi = 0;
        for (j = 0; j < ORC_BLOCK; j++) {
            i = k * ORC_BLOCK + j;
            if (i < n) {
                if (v[i] < lo)
                    lo = v[i];
                if (v[i] > hi)
                    hi = v[i];
            }
        }
        mn[k] = lo;
        b[k] = (uint8_t)orc_bitlen((uint64_t)hi - lo);
        sum_b += b[k];
    }
    packed_size = orc_fr_size(nb, sum_b);
    raw_size = orc_fq_raw_size(n);
    packed = (n > 0) && (packed_size < raw_size);
    size = packed ? packed_size : raw_size;
    *out_bytes = size;
    if (size > cap) {
        free(b);
        free(mn);
        return ORC_ENOSPC;
    }
    memset(out, 0, size);
    if (!packed) {
        put_u32(out + 0, ORC_MAGIC_FOR_RAW);
        put_u32(out + 4, (uint32_t)n);
        put_u32(out + 8, 0u);
        put_u32(out + 12, (uint32_t)n);
        for (i = 0; i < n; i++)
            put_u32(out + 16u + 4u * i, v[i]);
        free(b);
        free(mn);
        return ORC_OK;
    }
    put_u32(out + 0, ORC_MAGIC_FOR);
    put_u32(out + 4, (uint32_t)n);
    put_u32(out + 8, (uint32_t)nb);
    put_u32(out + 12, (uint32_t)(4u * sum_b));
    for (k = 0; k < nb; k++) {
        put_u32(out + 16u + 4u * k, mn[k]);
        out[16u + 4u * nb + k] = b[k];
    }
    bit0 = 8u * (16u + pad16(5u * nb));
    for (k = 0; k < nb; k++) {
        for (j = 0; j < ORC_BLOCK; j++) {
            uint64_t off = 0;
            i = k * ORC_BLOCK + j;
            if (i < n)
                off = (uint64_t)v[i] - mn[k];
            for (t = 0; t < b[k]; t++)
                if ((off >> t) & 1u)
                    set_bit(out, bit0 + j * b[k] + t);
        }
        bit0 += 128u * b[k];
    }
    free(b);
    free(mn);
    return ORC_OK;
}

/* Inverse of orc_fr_encode.  Rejects (ORC_ECORRUPT): unknown magic, nb != ceil(n/128), a width
 * > 32, payload_words != 4*sum(b), in_bytes != the layout's size, nonzero pads or padding slots,
 * and values above 2^32 - 1.  n > cap gives ORC_ENOSPC with *n_out = n. */
int orc_fr_decode(const uint8_t *in, uint64_t in_bytes, uint32_t *out, uint64_t cap, uint64_t *n_out)
{
    uint32_t magic;
    uint64_t n, nb, words, k, j, t, i, sum_b = 0, payload, bit0;

    *n_out = 0;
    if (in_bytes < 16u)
        return ORC_ECORRUPT;
    magic = get_u32(in);
    n = get_u32(in + 4);
    nb = get_u32(in + 8);
    words = get_u32(in + 12);
    if (magic == ORC_MAGIC_FOR_RAW) {
        if (nb != 0u || words != n || in_bytes != orc_fq_raw_size(n))
            return ORC_ECORRUPT;
        for (i = 16u + 4u * n; i < in_bytes; i++)
            if (in[i] != 0u)
                return ORC_ECORRUPT;
        *n_out = n;
        if (n > cap)
            return ORC_ENOSPC;
        for (i = 0; i < n; i++)
            out[i] = get_u32(in + 16u + 4u * i);
        return ORC_OK;
    }
    if (magic != ORC_MAGIC_FOR || nb != (n + ORC_BLOCK - 1u) / ORC_BLOCK || in_bytes < 16u + pad16(5u * nb))
        return ORC_ECORRUPT;
    for (k = 0; k < nb; k++) {
        if (in[16u + 4u * nb + k] > 32u)
            return ORC_ECORRUPT;
        sum_b += in[16u + 4u * nb + k];
    }
    payload = 16u + pad16(5u * nb);
    if (words != 4u * sum_b || in_bytes != orc_fr_size(nb, sum_b))
        return ORC_ECORRUPT;
    for (i = 16u + 5u * nb; i < payload; i++)
        if (in[i] != 0u)
            return ORC_ECORRUPT;
    *n_out = n;
    if (n > cap)
        return ORC_ENOSPC;
    bit0 = 8u * payload;
    for (k = 0; k < nb; k++) {
        uint32_t bk = in[16u + 4u * nb + k];
        uint64_t base = get_u32(in + 16u + 4u * k);
        for (j = 0; j < ORC_BLOCK; j++) {
            uint64_t off = 0;
            for (t = 0; t < bk; t++)
                off |= (uint64_t)get_bit(in, bit0 + j * bk + t) << t;
            i = k * ORC_BLOCK + j;
            if (i >= n) {
                if (off != 0u)
                    return ORC_ECORRUPT;
                continue;
            }
            if (base + off > 0xFFFFFFFFu)
                return ORC_ECORRUPT;
            out[i] = (uint32_t)(base + off);
        }
        bit0 += 128u * bk;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ bitmap codec "FB"
 *
 * A bitmap of N bits in u64 words (bit i is bit i%64 of word i/64).  P = number of set bits.
 * If 2P <= N the set positions (mode SET), else the clear positions below N (mode CLEAR), are
 * coded as an FQ stream behind the header {u32 "FBM1", u32 mode, u64 N}.  If that is not
 * strictly smaller than the raw form (header + the words, tail bits cleared, zero pad to
 * 16 bytes), the raw form (mode RAW) is written.
 */

uint64_t orc_fb_raw_size(uint64_t nbits) { return 16u + pad16(8u * ((nbits + 63u) / 64u)); }

static uint32_t word_bit(const uint64_t *words, uint64_t i) { return (uint32_t)((words[i / 64u] >> (i % 64u)) & 1u); }

int orc_fb_encode(const uint64_t *words, uint64_t nbits, uint8_t *out, uint64_t cap, uint64_t *out_bytes)
{
    uint64_t i, p = 0, count = 0, inner_bytes = 0, raw_size, nwords;
    uint32_t mode, want;
    uint32_t *pos;
    uint8_t *inner;
    int st;

    *out_bytes = 0;
    if (nbits > 0x100000000ull)
        return ORC_EINVAL;
    nwords = (nbits + 63u) / 64u;
    for (i = 0; i < nbits; i++)
        p += word_bit(words, i);
    mode = (2u * p <= nbits) ? ORC_FB_SET : ORC_FB_CLEAR;
    want = (mode == ORC_FB_SET) ? 1u : 0u;

    pos = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nbits ? nbits : 1u));
    if (!pos)
        return ORC_ENOMEM;
    for (i = 0; i < nbits; i++)
        if (word_bit(words, i) == want)
            pos[count++] = (uint32_t)i;
    inner = (uint8_t *)malloc((size_t)orc_fq_raw_size(count));
    if (!inner) {
        free(pos);
        return ORC_ENOMEM;
    }
    st = orc_fq_encode(pos, count, inner, orc_fq_raw_size(count), &inner_bytes);
    free(pos);
    if (st != ORC_OK) {
        free(inner);
        return st;
    }

    raw_size = orc_fb_raw_size(nbits);
    if (16u + inner_bytes >= raw_size) {
        *out_bytes = raw_size;
        if (raw_size > cap) {
            free(inner);
            return ORC_ENOSPC;
        }
        memset(out, 0, raw_size);
        put_u32(out, ORC_MAGIC_BITMAP);
        put_u32(out + 4, ORC_FB_RAW);
        put_u64(out + 8, nbits);
        for (i = 0; i < nbits; i++)
            if (word_bit(words, i))
                set_bit(out + 16, i);
        free(inner);
        (void)nwords;
        return ORC_OK;
    }
    *out_bytes = 16u + inner_bytes;
    if (*out_bytes > cap) {
        free(inner);
        return ORC_ENOSPC;
    }
    put_u32(out, ORC_MAGIC_BITMAP);
    put_u32(out + 4, mode);
    put_u64(out + 8, nbits);
    memcpy(out + 16, inner, (size_t)inner_bytes);
    free(inner);
    return ORC_OK;
}

/* Inverse of orc_fb_encode into words[0 .. ceil(nbits/64)).  The header's N must equal nbits;
 * every position must be below N; a raw stream must have zero tail bits and zero padding. */
int orc_fb_decode(const uint8_t *in, uint64_t in_bytes, uint64_t *words, uint64_t nbits)
{
    uint64_t nwords = (nbits + 63u) / 64u, i, count = 0;
    uint32_t mode;
    uint32_t *pos;
    int st;

    if (in_bytes < 16u || get_u32(in) != ORC_MAGIC_BITMAP || get_u64(in + 8) != nbits)
        return ORC_ECORRUPT;
    mode = get_u32(in + 4);
    if (mode == ORC_FB_RAW) {
        if (in_bytes != orc_fb_raw_size(nbits))
            return ORC_ECORRUPT;
        for (i = nbits; i < 8u * (in_bytes - 16u); i++)
            if (get_bit(in + 16, i))
                return ORC_ECORRUPT;
        for (i = 0; i < nwords; i++)
            words[i] = 0;
        for (i = 0; i < nbits; i++)
            if (get_bit(in + 16, i))
                words[i / 64u] |= (uint64_t)1u << (i % 64u);
        return ORC_OK;
    }
    if (mode != ORC_FB_SET && mode != ORC_FB_CLEAR)
        return ORC_ECORRUPT;
    pos = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nbits ? nbits : 1u));
    if (!pos)
        return ORC_ENOMEM;
    st = orc_fq_decode(in + 16, in_bytes - 16u, pos, nbits, &count);
    if (st != ORC_OK) {
        free(pos);
        return st == ORC_ENOSPC ? ORC_ECORRUPT : st;
    }
    if (count > 0 && (uint64_t)pos[count - 1u] >= nbits) {
        free(pos);
        return ORC_ECORRUPT;
    }
    for (i = 0; i < nwords; i++)
        words[i] = 0;
    if (mode == ORC_FB_CLEAR)
        for (i = 0; i < nbits; i++)
            words[i / 64u] |= (uint64_t)1u << (i % 64u);
    for (i = 0; i < count; i++) {
        uint64_t q = pos[i];
        if (mode == ORC_FB_SET)
            words[q / 64u] |= (uint64_t)1u << (q % 64u);
        else
            words[q / 64u] &= ~((uint64_t)1u << (q % 64u));
    }
    free(pos);
    return ORC_OK;
}

/* ------------------------------------------------------------------ BFS
 *
 * Level-synchronous BFS from root over an undirected graph in CSR (offsets[n+1], cols[m]):
 * depth[v] = hop distance from root, -1 if unreachable; parent[v] = the vertex that discovered
 * v first in FIFO order, parent[root] = root, UINT32_MAX if unreachable.  This is the
 * frontier / visited-list recurrence of the thesis' BFS (f <- A (x) f masked by not-visited,
 * visited <- visited + f), run as the textbook FIFO queue.
 */
int orc_bfs(uint64_t n, const int64_t *offsets, const uint32_t *cols, uint32_t root, int32_t *depth,
            uint32_t *parent)
{
    uint32_t *queue;
    uint64_t head = 0, tail = 0, v;
    int64_t e;

    if (root >= n)
        return ORC_EINVAL;
    queue = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1u));
    if (!queue)
        return ORC_ENOMEM;
    for (v = 0; v < n; v++) {
        depth[v] = -1;
        parent[v] = 0xFFFFFFFFu;
    }
    depth[root] = 0;
    parent[root] = root;
    queue[tail++] = root;
    while (head < tail) {
        uint32_t u = queue[head++];
        for (e = offsets[u]; e < offsets[u + 1]; e++) {
            uint32_t w = cols[e];
            if (depth[w] == -1) {
                depth[w] = depth[u] + 1;
                parent[w] = u;
                queue[tail++] = w;
            }
        }
    }
    free(queue);
    return ORC_OK;
}

/* BFS-tree validation of (depth, parent) for root; returns 0 if valid, else the number of the
 * first rule that fails:
 *   1  root: depth[root] = 0 and parent[root] = root; no other vertex has depth 0; depth >= -1
 *   2  every reached v != root: parent[v] < n, (parent[v], v) is an edge of the graph and
 *      depth[parent[v]] = depth[v] - 1
 *   3  every edge (u, w): both endpoints unreached, or both reached with |depth u - depth w| <= 1
 *      (so the reached set is closed under edges: it is root's connected component)
 *   4  every unreached v has parent[v] = UINT32_MAX
 */
int orc_validate(uint64_t n, const int64_t *offsets, const uint32_t *cols, uint32_t root, const int32_t *depth,
                 const uint32_t *parent)
{
    uint64_t v;
    int64_t e;

    if (root >= n || depth[root] != 0 || parent[root] != root)
        return 1;
    for (v = 0; v < n; v++) {
        if (depth[v] < -1)
            return 1;
        if (depth[v] == 0 && v != root)
            return 1;
    }
    for (v = 0; v < n; v++) {
        uint32_t p;
        int found = 0;
        if (v == root || depth[v] < 0)
            continue;
        p = parent[v];
        if ((uint64_t)p >= n)
            return 2;
        for (e = offsets[v]; e < offsets[v + 1]; e++) /* undirected: p is a neighbour of v */
            if (cols[e] == p)
                found = 1;
        if (!found || depth[p] != depth[v] - 1)
            return 2;
    }
    for (v = 0; v < n; v++) {
        for (e = offsets[v]; e < offsets[v + 1]; e++) {
            int32_t a = depth[v], c = depth[cols[e]];
            if ((a < 0) != (c < 0))
                return 3;
            if (a >= 0 && (a - c > 1 || c - a > 1))
                return 3;
        }
    }
    for (v = 0; v < n; v++)
        if (depth[v] < 0 && parent[v] != 0xFFFFFFFFu)
            return 4;
    return 0;
}

/* Edges examined by a bottom-up sweep that expands level d (frontier F_d = {depth == d}):
 * every vertex w not yet visited (depth[w] == -1 or depth[w] > d) scans its adjacency in CSR
 * order and stops at the first neighbour in F_d; it examines (index of that neighbour + 1)
 * edges, or deg(w) when none is found.  Direction optimisation, sec. 3.1. */
uint64_t orc_bu_examined(uint64_t n, const int64_t *offsets, const uint32_t *cols, const int32_t *depth, int32_t d)
{
    uint64_t v, total = 0;
    int64_t e;

    for (v = 0; v < n; v++) {
        if (depth[v] != -1 && depth[v] <= d)
            continue;
        for (e = offsets[v]; e < offsets[v + 1]; e++) {
            total++;
            if (depth[cols[e]] == d)
                break;
        }
    }
    return total;
}
