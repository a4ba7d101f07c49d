/*
 * CPU oracle for the FNR impulse filter of "A Novel Approach to Fast Image
 * Filtering Algorithm of Infrared Images based on Intro Sort Algorithm"
 * (arXiv 1201.3972).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA library is checked against. Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg load it; the library never calls it, and
 * the two share no code, header, table or helper.
 *
 * What it computes, step by step in the paper's order (Sec. 3.3 and 3.4):
 *   1. S_xy: the k x k window around p(x, y), centre included, gathered
 *      row-major as in the paper's 3x3 listing (Sec. 3.3).
 *   2. g_max = max S_xy and g_min = min S_xy (Eq. 3a, 3b).
 *   3. p(x, y) is noisy iff g(x, y) == g_min or g(x, y) == g_max (Sec. 3.3,
 *      step 2); otherwise it is a signal pixel.
 *   4. A noisy pixel is replaced by the median gray level g_m of S_xy, found
 *      by sorting S_xy with introsort (quicksort that falls back to heapsort
 *      past a depth limit, Sec. 3.4, Eq. 4); signal pixels are left as they are.
 *
 * Readings where the paper is silent:
 *   - border: replicate (clamp to edge); every pixel, border included, gets
 *     the full n = k*k window (Table 1 counts a min/max evaluation for every
 *     one of the 364 x 244 pixels);
 *   - every window reads the unfiltered input frame (one non-recursive pass);
 *   - ties flag (the equality test of step 3 is taken literally);
 *   - k is odd, so n is odd and g_m is the element of rank m = (n-1)/2
 *     (0-based) of the sorted window.
 *
 * Pixels are 8-bit (esize 1) or 16-bit (esize 2) unsigned integers in a
 * row-pitched buffer (pitch in bytes). Comparison is plain unsigned integer
 * comparison, so the result does not depend on how many bits are used.
 */
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------------ */
/* Introsort (Sec. 3.4, Eq. 4), written out plainly.                         */
/* ------------------------------------------------------------------------ */

static void swap_u32(uint32_t *a, uint32_t *b) { uint32_t t = *a; *a = *b; *b = t; }

static void insertion_sort(uint32_t *a, long n)
{
    for (long i = 1; i < n; i++) {
        uint32_t v = a[i];
        long j = i - 1;
        while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; j--; }
        a[j + 1] = v;
    }
}

/* Max-heap sift-down over a[0..end). */
static void sift_down(uint32_t *a, long root, long end)
{
    for (;;) {
        long child = 2 * root + 1;
        if (child >= end) return;
        if (child + 1 < end && a[child + 1] > a[child]) child++;
        if (a[root] >= a[child]) return;
        swap_u32(&a[root], &a[child]);
        root = child;
    }
}

static void heap_sort(uint32_t *a, long n)
{
    for (long i = n / 2 - 1; i >= 0; i--) sift_down(a, i, n);
    for (long end = n - 1; end > 0; end--) {
        swap_u32(&a[0], &a[end]);
        sift_down(a, 0, end);
    }
}

/* Quicksort with a median-of-three pivot and Hoare partitioning; once the
 * recursion depth budget is spent the remaining range is heapsorted, and
 * ranges of at most 16 elements are finished by insertion sort. */
static void intro_rec(uint32_t *a, long n, int depth)
{
    while (n > 16) {
        if (depth == 0) { heap_sort(a, n); return; }
        depth--;
        long mid = n / 2;
        /* order a[0] <= a[mid] <= a[n-1]; the pivot is the middle value */
        if (a[mid] < a[0]) swap_u32(&a[mid], &a[0]);
        if (a[n - 1] < a[0]) swap_u32(&a[n - 1], &a[0]);
        if (a[n - 1] < a[mid]) swap_u32(&a[n - 1], &a[mid]);
        uint32_t pivot = a[mid];
        long i = -1, j = n;
        for (;;) {
            do { i++; } while (a[i] < pivot);
            do { j--; } while (a[j] > pivot);
            if (i >= j) break;
            swap_u32(&a[i], &a[j]);
        }
        /* a[0..j] <= pivot <= a[j+1..n-1], both parts non-empty */
        intro_rec(a + j + 1, n - j - 1, depth);
        n = j + 1;
    }
    insertion_sort(a, n);
}

static int floor_log2(long n)
{
    int l = 0;
    while (n > 1) { n >>= 1; l++; }
    return l;
}

/* Sort a[0..n) ascending. depth_limit < 0 selects the usual 2*floor(log2 n);
 * 0 forces the heapsort fallback at once (used by the tests to exercise it). */
void oracle_introsort(uint32_t *a, long n, int depth_limit)
{
    if (n < 2) return;
    int depth = depth_limit < 0 ? 2 * floor_log2(n) : depth_limit;
    intro_rec(a, n, depth);
}

/* ------------------------------------------------------------------------ */
/* The filter.                                                               */
/* ------------------------------------------------------------------------ */

static uint32_t load_px(const unsigned char *base, long long pitch, int esize, int y, int x)
{
    const unsigned char *row = base + (long long)y * pitch;
    if (esize == 1) return row[x];
    uint16_t v;
    memcpy(&v, row + 2 * (long long)x, 2);
    return v;
}

static void store_px(unsigned char *base, long long pitch, int esize, int y, int x, uint32_t v)
{
    unsigned char *row = base + (long long)y * pitch;
    if (esize == 1) { row[x] = (unsigned char)v; return; }
    uint16_t s = (uint16_t)v;
    memcpy(row + 2 * (long long)x, &s, 2);
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Border readings (the paper is silent; replicate is the default):
 *   0 replicate: clamp to the nearest edge pixel;
 *   1 mirror: reflect about the edge pixel without repeating it (d c b | a b c d | c b a),
 *     periodic with period 2(n-1) for windows wider than the frame;
 *   2 zero: pixels outside the frame read as 0.
 * Returns the in-frame index to read, or -1 for "reads 0". */
static int border_index(int i, int n, int mode)
{
    if (i >= 0 && i < n) return i;
    if (mode == 2) return -1;
    if (mode == 1) {
        if (n == 1) return 0;
        int period = 2 * (n - 1);
        int j = i % period;
        if (j < 0) j += period;
        return j < n ? j : period - j;
    }
    return clampi(i, 0, n - 1);
}

/* Rows [y0, y1) of the output. w is scratch for n = k*k values. */
static long long fnr_rows_b(const unsigned char *in, long long in_pitch,
                            unsigned char *out, long long out_pitch,
                            int H, int W, int esize, int k, int y0, int y1, uint32_t *w, int border);

static long long fnr_rows(const unsigned char *in, long long in_pitch,
                          unsigned char *out, long long out_pitch,
                          int H, int W, int esize, int k, int y0, int y1, uint32_t *w)
{
    return fnr_rows_b(in, in_pitch, out, out_pitch, H, W, esize, k, y0, y1, w, 0);
}

static long long fnr_rows_b(const unsigned char *in, long long in_pitch,
                            unsigned char *out, long long out_pitch,
                            int H, int W, int esize, int k, int y0, int y1, uint32_t *w, int border)
{
    const int r = (k - 1) / 2;
    const int n = k * k;
    const int m = (n - 1) / 2;
    long long flagged = 0;
    for (int y = y0; y < y1; y++) {
        for (int x = 0; x < W; x++) {
            /* 1. S_xy, centre included, row-major, border per the reading in use */
            int i = 0;
            for (int dy = -r; dy <= r; dy++) {
                int yy = border_index(y + dy, H, border);
                for (int dx = -r; dx <= r; dx++) {
                    int xx = border_index(x + dx, W, border);
                    w[i++] = (yy < 0 || xx < 0) ? 0u : load_px(in, in_pitch, esize, yy, xx);
                }
            }
            /* 2. g_max and g_min (Eq. 3a, 3b) */
            uint32_t gmin = w[0], gmax = w[0];
            for (i = 1; i < n; i++) {
                if (w[i] < gmin) gmin = w[i];
                if (w[i] > gmax) gmax = w[i];
            }
            /* 3. noisy iff g(x,y) equals g_min or g_max */
            uint32_t g = load_px(in, in_pitch, esize, y, x);
            uint32_t v = g;
            if (g == gmin || g == gmax) {
                /* 4. median of S_xy by introsort */
                oracle_introsort(w, n, -1);
                v = w[m];
                flagged++;
            }
            store_px(out, out_pitch, esize, y, x, v);
        }
    }
    return flagged;
}

static int args_ok(const void *in, long long in_pitch, const void *out, long long out_pitch,
                   int H, int W, int esize, int k)
{
    if (!in || !out) return 0;
    if (H < 1 || W < 1) return 0;
    if (esize != 1 && esize != 2) return 0;
    if (k < 1 || (k % 2) == 0 || k > 255) return 0;
    if (in_pitch < (long long)W * esize || out_pitch < (long long)W * esize) return 0;
    return 1;
}

/* One frame, one thread. Returns the number of noisy (flagged) pixels, i.e.
 * the number of medians taken (the "sort times" of Table 1), or -1 for bad
 * arguments. in and out must not overlap. */
long long oracle_fnr(const void *in, long long in_pitch, void *out, long long out_pitch,
                     int H, int W, int esize, int k)
{
    if (!args_ok(in, in_pitch, out, out_pitch, H, W, esize, k)) return -1;
    uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)k * (size_t)k);
    if (!w) return -1;
    long long f = fnr_rows((const unsigned char *)in, in_pitch, (unsigned char *)out, out_pitch,
                           H, W, esize, k, 0, H, w);
    free(w);
    return f;
}

/* oracle_fnr with a border reading other than replicate (see border_index). */
long long oracle_fnr_border(const void *in, long long in_pitch, void *out, long long out_pitch,
                            int H, int W, int esize, int k, int border)
{
    if (!args_ok(in, in_pitch, out, out_pitch, H, W, esize, k) || border < 0 || border > 2) return -1;
    uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)k * (size_t)k);
    if (!w) return -1;
    long long f = fnr_rows_b((const unsigned char *)in, in_pitch, (unsigned char *)out, out_pitch,
                             H, W, esize, k, 0, H, w, border);
    free(w);
    return f;
}

/* `count` frames of identical shape stored back to back (each H*pitch bytes). */
long long oracle_fnr_stack(const void *in, void *out, long long pitch, int count,
                           int H, int W, int esize, int k)
{
    long long total = 0;
    for (int i = 0; i < count; i++) {
        long long off = (long long)i * H * pitch;
        long long f = oracle_fnr((const unsigned char *)in + off, pitch,
                                 (unsigned char *)out + off, pitch, H, W, esize, k);
        if (f < 0) return -1;
        total += f;
    }
    return total;
}

/* The standard median filter the paper compares FNR with (Sec. 2, Table 1,
 * "MF"): every pixel, noisy or not, is replaced by the median of S_xy,
 * found the same way (introsort, element (n-1)/2). Returns the number of
 * medians taken (H*W), or -1 for bad arguments. */
long long oracle_median_filter(const void *in, long long in_pitch, void *out, long long out_pitch,
                               int H, int W, int esize, int k)
{
    if (!args_ok(in, in_pitch, out, out_pitch, H, W, esize, k)) return -1;
    const int r = (k - 1) / 2;
    const int n = k * k;
    uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    if (!w) return -1;
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            int i = 0;
            for (int dy = -r; dy <= r; dy++) {
                int yy = clampi(y + dy, 0, H - 1);
                for (int dx = -r; dx <= r; dx++)
                    w[i++] = load_px((const unsigned char *)in, in_pitch, esize, yy, clampi(x + dx, 0, W - 1));
            }
            oracle_introsort(w, n, -1);
            store_px((unsigned char *)out, out_pitch, esize, y, x, w[(n - 1) / 2]);
        }
    }
    free(w);
    return (long long)H * W;
}

/* The directional detector, an option beside Eq. 3a/3b. Fig. 1 (its image
 * is missing) compares the centre of a 3x3 window with its two neighbours
 * along each direction, and Sec. 3 rests on the gray level of a signal pixel
 * varying monotonically over an object's surface (Eq. 1 and 2). Reading:
 * p(x, y) is a signal pixel iff along at least one of the four lines through
 * it (horizontal, vertical, the two diagonals) g(x, y) lies strictly between
 * its two neighbours at distance one; otherwise it is noisy and takes the
 * median of the k x k window S_xy (Sec. 3.4). Neighbours and window are read
 * under the same border reading. Returns the number of noisy pixels, or -1
 * for bad arguments. */
long long oracle_fnr_directional(const void *in, long long in_pitch, void *out, long long out_pitch,
                                 int H, int W, int esize, int k, int border)
{
    if (!args_ok(in, in_pitch, out, out_pitch, H, W, esize, k) || border < 0 || border > 2) return -1;
    /* one end of each line; the other end is the opposite offset */
    static const int line_dy[4] = {0, -1, -1, -1};
    static const int line_dx[4] = {-1, 0, -1, 1};
    const unsigned char *src = (const unsigned char *)in;
    const int r = (k - 1) / 2;
    const int n = k * k;
    uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    if (!w) return -1;
    long long flagged = 0;
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            uint32_t g = load_px(src, in_pitch, esize, y, x);
            int monotone = 0;
            for (int d = 0; d < 4; d++) {
                int ya = border_index(y + line_dy[d], H, border), xa = border_index(x + line_dx[d], W, border);
                int yb = border_index(y - line_dy[d], H, border), xb = border_index(x - line_dx[d], W, border);
                uint32_t a = (ya < 0 || xa < 0) ? 0u : load_px(src, in_pitch, esize, ya, xa);
                uint32_t b = (yb < 0 || xb < 0) ? 0u : load_px(src, in_pitch, esize, yb, xb);
                if ((a < g && g < b) || (b < g && g < a)) monotone = 1;
            }
            uint32_t v = g;
            if (!monotone) {
                int i = 0;
                for (int dy = -r; dy <= r; dy++) {
                    int yy = border_index(y + dy, H, border);
                    for (int dx = -r; dx <= r; dx++) {
                        int xx = border_index(x + dx, W, border);
                        w[i++] = (yy < 0 || xx < 0) ? 0u : load_px(src, in_pitch, esize, yy, xx);
                    }
                }
                oracle_introsort(w, n, -1);
                v = w[(n - 1) / 2];
                flagged++;
            }
            store_px((unsigned char *)out, out_pitch, esize, y, x, v);
        }
    }
    free(w);
    return flagged;
}

/* Same result, rows split into contiguous bands over `threads` POSIX threads
 * (used only to time the oracle on all host cores). */
typedef struct {
    const unsigned char *in; long long in_pitch;
    unsigned char *out; long long out_pitch;
    int H, W, esize, k, y0, y1;
    long long flagged;
    int failed;
} band_job;

static void *band_main(void *p)
{
    band_job *j = (band_job *)p;
    uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)j->k * (size_t)j->k);
    if (!w) { j->failed = 1; return NULL; }
    j->flagged = fnr_rows(j->in, j->in_pitch, j->out, j->out_pitch, j->H, j->W, j->esize, j->k,
                          j->y0, j->y1, w);
    free(w);
    return NULL;
}

long long oracle_fnr_mt(const void *in, long long in_pitch, void *out, long long out_pitch,
                        int H, int W, int esize, int k, int threads)
{
    if (!args_ok(in, in_pitch, out, out_pitch, H, W, esize, k)) return -1;
    if (threads < 1) threads = 1;
    if (threads > H) threads = H;
    if (threads > 256) threads = 256;
    band_job jobs[256];
    pthread_t tids[256];
    int started[256];
    for (int t = 0; t < threads; t++) {
        jobs[t].in = (const unsigned char *)in; jobs[t].in_pitch = in_pitch;
        jobs[t].out = (unsigned char *)out; jobs[t].out_pitch = out_pitch;
        jobs[t].H = H; jobs[t].W = W; jobs[t].esize = esize; jobs[t].k = k;
        jobs[t].y0 = (int)((long long)H * t / threads);
        jobs[t].y1 = (int)((long long)H * (t + 1) / threads);
        jobs[t].flagged = 0; jobs[t].failed = 0;
        started[t] = pthread_create(&tids[t], NULL, band_main, &jobs[t]) == 0;
        if (!started[t]) band_main(&jobs[t]);
    }
    long long total = 0;
    int failed = 0;
    for (int t = 0; t < threads; t++) {
        if (started[t]) pthread_join(tids[t], NULL);
        total += jobs[t].flagged;
        failed |= jobs[t].failed;
    }
    return failed ? -1 : total;
}
