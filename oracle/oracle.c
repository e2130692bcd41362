/*
 * Plain FP64 CPU oracle for decentralized ADMM tomography with quantized
 * messages (arXiv 2410.06106). TEST INFRASTRUCTURE ONLY: the test suite, the
 * smoke check and the benchmark's CPU-baseline leg load it; the CUDA library
 * shares no code with it.
 *
 * Written for readability, not speed: every operator entry is evaluated from
 * its geometric definition (Eq. 2), every algorithm step follows the paper's
 * order (Algorithms 2-5, Eq. 15-18 and 21-24). OpenMP only splits loops whose
 * iterations write disjoint outputs, so results do not depend on the thread
 * count.
 *
 * Readings where the paper is silent:
 *  - geometry conventions: see oracle.h;
 *  - Algorithm 2 is warm-started from u_m^k (zero only at k = 0);
 *  - Algorithm 3 acts on the rows of segment m and is warm-started from the
 *    owner's unquantized segment;
 *  - segments are contiguous row bands seg_row_ptr[m] .. seg_row_ptr[m+1];
 *  - messages travel along shortest paths of the node graph, one hop per
 *    iteration, relayed verbatim; the quantizer of a message is that of the
 *    first edge on the path (lowest-id parent on ties); a node's own segment
 *    uses its home quantizer; on a complete graph this is Eq. 23 exactly;
 *  - K-means: seeded initial centres at distinct values, ties to the lower
 *    centre, empty clusters keep their centre, FP32 decisions (the paper's
 *    images are 32-bit), FP64 centroid sums;
 *  - JPEG: per-segment min/max affine map to 8-bit samples, level shift 128,
 *    orthonormal 8x8 DCT-II, luminance table of ITU-T T.81 Annex K scaled by
 *    the IJG quality rule, rounding half away from zero, no entropy coding
 *    (it is lossless and changes no value).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_GOLDEN 0x9E3779B97F4A7C15ULL

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* geometry (Sec. 2.1, Eq. 1-4)                                        */
/* ------------------------------------------------------------------ */

void orc_trig(int n, const double* theta, double* c, double* s) {
    for (int a = 0; a < n; ++a) {
        double q = theta[a] / (0.5 * ORC_PI);
        double k = floor(q + 0.5);
        if (fabs(theta[a] - k * 0.5 * ORC_PI) < 1e-12) {
            long m = ((long)k % 4 + 4) % 4;
            c[a] = (m == 0) ? 1.0 : (m == 2) ? -1.0 : 0.0;
            s[a] = (m == 1) ? 1.0 : (m == 3) ? -1.0 : 0.0;
        } else {
            c[a] = cos(theta[a]);
            s[a] = sin(theta[a]);
        }
    }
}

/* Length of {x c + y s = t} inside [xc-1/2, xc+1/2] x [yc-1/2, yc+1/2].
 * The line is p(l) = (t c - l s, t s + l c), a unit-speed parametrisation;
 * clip l against the two slabs of the square. */
double orc_chord(double c, double s, double t, double xc, double yc) {
    double lo = -INFINITY, hi = INFINITY, w = 1.0;
    if (s == 0.0) { /* vertical line x = t c */
        double off = fabs(t * c - xc);
        if (off > 0.5) return 0.0;
        if (off == 0.5) w *= 0.5; /* on a pixel edge: split between the two pixels */
    } else {
        double l1 = (t * c - xc - 0.5) / s, l2 = (t * c - xc + 0.5) / s;
        lo = fmax(lo, fmin(l1, l2));
        hi = fmin(hi, fmax(l1, l2));
    }
    if (c == 0.0) { /* horizontal line y = t s */
        double off = fabs(t * s - yc);
        if (off > 0.5) return 0.0;
        if (off == 0.5) w *= 0.5;
    } else {
        double l1 = (yc - 0.5 - t * s) / c, l2 = (yc + 0.5 - t * s) / c;
        lo = fmax(lo, fmin(l1, l2));
        hi = fmin(hi, fmax(l1, l2));
    }
    return hi > lo ? w * (hi - lo) : 0.0;
}

/* Bins whose line can meet pixel (xc, yc): the square's projection onto the
 * ray normal is [tau0 - w, tau0 + w], w = (|c| + |s|) / 2. All other entries
 * of the column are exactly zero, so skipping them leaves the sums unchanged. */
static void bin_range(double c, double s, double xc, double yc, int B, int* b0, int* b1) {
    double w = 0.5 * (fabs(c) + fabs(s));
    double pc = xc * c + yc * s + 0.5 * (B - 1);
    int lo = (int)ceil(pc - w - 1e-9), hi = (int)floor(pc + w + 1e-9);
    *b0 = lo < 0 ? 0 : lo;
    *b1 = hi > B - 1 ? B - 1 : hi;
}

void orc_project(int N, int B, const double* c, const double* s, int nsel,
                 const int32_t* aidx, int batch, const double* img, double* sino) {
    const long n = (long)N * N;
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < nsel; ++q) {
        const int a = aidx[q];
        for (int bt = 0; bt < batch; ++bt)
            memset(sino + ((long)bt * nsel + q) * B, 0, sizeof(double) * B);
        for (int i = 0; i < N; ++i) {
            const double yc = 0.5 * (N - 1) - i;
            for (int j = 0; j < N; ++j) {
                const double xc = j - 0.5 * (N - 1);
                int b0, b1;
                bin_range(c[a], s[a], xc, yc, B, &b0, &b1);
                for (int b = b0; b <= b1; ++b) {
                    double w = orc_chord(c[a], s[a], b - 0.5 * (B - 1), xc, yc);
                    if (w == 0.0) continue;
                    for (int bt = 0; bt < batch; ++bt)
                        sino[((long)bt * nsel + q) * B + b] += w * img[bt * n + (long)i * N + j];
                }
            }
        }
    }
}

void orc_backproject(int N, int B, const double* c, const double* s, int nsel,
                     const int32_t* aidx, int batch, const double* sino, double* img) {
    const long n = (long)N * N;
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) {
        const int i = (int)(p / N), j = (int)(p % N);
        const double yc = 0.5 * (N - 1) - i, xc = j - 0.5 * (N - 1);
        for (int bt = 0; bt < batch; ++bt) {
            double acc = 0.0;
            for (int q = 0; q < nsel; ++q) {
                const int a = aidx[q];
                int b0, b1;
                bin_range(c[a], s[a], xc, yc, B, &b0, &b1);
                for (int b = b0; b <= b1; ++b) {
                    double w = orc_chord(c[a], s[a], b - 0.5 * (B - 1), xc, yc);
                    acc += w * sino[((long)bt * nsel + q) * B + b];
                }
            }
            img[bt * n + p] = acc;
        }
    }
}

void orc_project_rays(int N, int B, const double* c, const double* s, int nray,
                      const int32_t* ray_a, const int32_t* ray_b,
                      const double* img, double* out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < nray; ++r) {
        const int a = ray_a[r];
        const double t = ray_b[r] - 0.5 * (B - 1);
        double acc = 0.0;
        for (int i = 0; i < N; ++i) {
            const double yc = 0.5 * (N - 1) - i;
            for (int j = 0; j < N; ++j) {
                const double xc = j - 0.5 * (N - 1);
                /* same support test as bin_range, seen from the ray */
                double w = 0.5 * (fabs(c[a]) + fabs(s[a]));
                if (fabs(t - (xc * c[a] + yc * s[a])) > w + 1e-9) continue;
                acc += orc_chord(c[a], s[a], t, xc, yc) * img[(long)i * N + j];
            }
        }
        out[r] = acc;
    }
}

void orc_backproject_pixels(int N, int B, const double* c, const double* s,
                            int nsel, const int32_t* aidx, const double* sino,
                            int npix, const int32_t* pix, double* out) {
#pragma omp parallel for schedule(static)
    for (int q = 0; q < npix; ++q) {
        const int i = pix[q] / N, j = pix[q] % N;
        const double yc = 0.5 * (N - 1) - i, xc = j - 0.5 * (N - 1);
        double acc = 0.0;
        for (int k = 0; k < nsel; ++k) {
            const int a = aidx[k];
            int b0, b1;
            bin_range(c[a], s[a], xc, yc, B, &b0, &b1);
            for (int b = b0; b <= b1; ++b)
                acc += orc_chord(c[a], s[a], b - 0.5 * (B - 1), xc, yc) * sino[(long)k * B + b];
        }
        out[q] = acc;
    }
}

static double dot(const double* a, const double* b, long n) {
    double acc = 0.0;
    for (long i = 0; i < n; ++i) acc += a[i] * b[i];
    return acc;
}

double orc_opnorm_sq(int N, int B, const double* c, const double* s, int nsel,
                     const int32_t* aidx, int iters, uint64_t seed) {
    const long n = (long)N * N;
    double* x = (double*)malloc(sizeof(double) * n);
    double* y = (double*)malloc(sizeof(double) * (long)nsel * B);
    double* z = (double*)malloc(sizeof(double) * n);
    for (long i = 0; i < n; ++i)
        x[i] = (double)(orc_mix64(seed + (uint64_t)(i + 1) * ORC_GOLDEN) >> 11) * 0x1.0p-53;
    double lam = 0.0;
    for (int it = 0; it < iters; ++it) {
        double nx = sqrt(dot(x, x, n));
        for (long i = 0; i < n; ++i) x[i] /= nx;
        orc_project(N, B, c, s, nsel, aidx, 1, x, y);
        orc_backproject(N, B, c, s, nsel, aidx, 1, y, z);
        lam = dot(x, z, n); /* Rayleigh quotient of P^T P at unit x */
        memcpy(x, z, sizeof(double) * n);
    }
    free(x); free(y); free(z);
    return lam;
}

/* ------------------------------------------------------------------ */
/* counter-based generator                                             */
/* ------------------------------------------------------------------ */

uint64_t orc_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_kmeans_key(uint64_t seed, int slice, int owner, int iter) {
    uint64_t ctr = ((uint64_t)(uint32_t)slice << 48) ^ ((uint64_t)(uint32_t)owner << 32) ^
                   (uint64_t)(uint32_t)iter;
    return orc_mix64(seed ^ orc_mix64(ctr + ORC_GOLDEN));
}

/* ------------------------------------------------------------------ */
/* Algorithm 5: K-means on a vector                                    */
/* ------------------------------------------------------------------ */

#define ORC_KM_PROBES 64

void orc_kmeans(const float* v, int64_t n, int k, int iters, uint64_t key,
                uint8_t* codes, float* cent, float* deq, double* obj) {
    /* initial centres: the values at k seeded indices; an index whose value is
     * already a centre moves on to the next index (at most ORC_KM_PROBES
     * times, then the repeated value is kept) */
    for (int j = 0; j < k; ++j) {
        uint64_t idx = orc_mix64(key + (uint64_t)(j + 1) * ORC_GOLDEN) % (uint64_t)n;
        float pick = v[idx];
        for (int p = 0; p < ORC_KM_PROBES; ++p) {
            float cand = v[(idx + (uint64_t)p) % (uint64_t)n];
            int dup = 0;
            for (int q = 0; q < j; ++q) dup |= (cent[q] == cand);
            if (!dup) { pick = cand; break; }
        }
        cent[j] = pick;
    }
    for (int j = 1; j < k; ++j) { /* ascending order */
        float t = cent[j];
        int q = j - 1;
        while (q >= 0 && cent[q] > t) { cent[q + 1] = cent[q]; --q; }
        cent[q + 1] = t;
    }

    double* sum = (double*)calloc((size_t)k, sizeof(double));
    int64_t* cnt = (int64_t*)calloc((size_t)k, sizeof(int64_t));
    for (int t = 0; t <= iters; ++t) {
        /* assignment: nearest centre by FP32 distance, ties to the lower index */
        double J = 0.0;
        for (int j = 0; j < k; ++j) { sum[j] = 0.0; cnt[j] = 0; }
        for (int64_t i = 0; i < n; ++i) {
            int best = 0;
            float bd = fabsf(v[i] - cent[0]);
            for (int j = 1; j < k; ++j) {
                float d = fabsf(v[i] - cent[j]);
                if (d < bd) { bd = d; best = j; }
            }
            codes[i] = (uint8_t)best;
            double e = (double)v[i] - (double)cent[best];
            J += e * e;
            sum[best] += (double)v[i];
            cnt[best] += 1;
        }
        if (obj) obj[t] = J;
        if (t == iters) break;
        /* update: each centre moves to the mean of its members */
        for (int j = 0; j < k; ++j)
            if (cnt[j] > 0) cent[j] = (float)(sum[j] / (double)cnt[j]);
    }
    for (int64_t i = 0; i < n; ++i) deq[i] = cent[codes[i]];
    free(sum);
    free(cnt);
}

/* ------------------------------------------------------------------ */
/* JPEG-style codec (Sec. 2.7, "standard JPEG")                        */
/* ------------------------------------------------------------------ */

/* ITU-T T.81 (1992) Annex K, Table K.1: luminance quantization table,
 * natural (row-major) order, row = vertical frequency. */
static const int ORC_JPEG_LUMA[64] = {
    16, 11, 10, 16, 24, 40, 51, 61,
    12, 12, 14, 19, 26, 58, 60, 55,
    14, 13, 16, 24, 40, 57, 69, 56,
    14, 17, 22, 29, 51, 87, 80, 62,
    18, 22, 37, 56, 68, 109, 103, 77,
    24, 35, 55, 64, 81, 104, 113, 92,
    49, 64, 78, 87, 103, 121, 120, 101,
    72, 92, 95, 98, 112, 100, 103, 99};

void orc_jpeg_qtable(int quality, int32_t* qt) {
    if (quality < 1) quality = 1;
    if (quality > 100) quality = 100;
    int scale = quality < 50 ? 5000 / quality : 200 - 2 * quality; /* IJG rule */
    for (int i = 0; i < 64; ++i) {
        long v = ((long)ORC_JPEG_LUMA[i] * scale + 50) / 100;
        qt[i] = (int32_t)(v < 1 ? 1 : v > 255 ? 255 : v);
    }
}

/* Weight of sample (i, j) in coefficient (p, q) of the orthonormal 2-D
 * DCT-II: 1/4 C(p) C(q) cos((2i+1) p pi/16) cos((2j+1) q pi/16), C(0) =
 * 1/sqrt(2). When p and q are both 0 or 4 the weight is exactly +-1/8
 * (cos((2i+1) pi/4) = +-1/sqrt(2)); it is used exactly, so that these four
 * coefficients (and image values built from them alone) are exact multiples
 * of 1/8 and their rounding ties are decided by the rounding rule. */
static int rational_freq(int p) { return p == 0 || p == 4; }

static double half_sign(int i, int p) { /* sign of cos((2i+1) p pi/16), p in {0, 4} */
    if (p == 0) return 1.0;
    const int m = (2 * i + 1) % 8; /* (2i+1) pi/4 modulo 2 pi */
    return (m == 1 || m == 7) ? 1.0 : -1.0;
}

static double dct_weight(int p, int q, int i, int j) {
    if (rational_freq(p) && rational_freq(q)) return 0.125 * half_sign(i, p) * half_sign(j, q);
    const double cp = p == 0 ? 1.0 / sqrt(2.0) : 1.0, cq = q == 0 ? 1.0 / sqrt(2.0) : 1.0;
    return 0.25 * cp * cq * cos((2 * i + 1) * p * ORC_PI / 16.0) * cos((2 * j + 1) * q * ORC_PI / 16.0);
}

/* F[p][q] = sum_i sum_j f[i][j] w(p, q, i, j) */
void orc_dct8x8(const double* in, double* out) {
    for (int p = 0; p < 8; ++p)
        for (int q = 0; q < 8; ++q) {
            double acc = 0.0;
            for (int i = 0; i < 8; ++i)
                for (int j = 0; j < 8; ++j) acc += in[i * 8 + j] * dct_weight(p, q, i, j);
            out[p * 8 + q] = acc;
        }
}

/* f[i][j] = sum_p sum_q F[p][q] w(p, q, i, j) (the transform is orthonormal) */
void orc_idct8x8(const double* in, double* out) {
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            double acc = 0.0;
            for (int p = 0; p < 8; ++p)
                for (int q = 0; q < 8; ++q) acc += in[p * 8 + q] * dct_weight(p, q, i, j);
            out[i * 8 + j] = acc;
        }
}

/* ---------------------------------------------------------------------
 * Baseline sequential Huffman coding of quantized 8x8 blocks (ITU-T T.81,
 * Annex F.1.2: DC differences by category + extra bits, AC run/size
 * symbols with ZRL and EOB, zig-zag order of Figure A.6), with the example
 * luminance tables of Annex K (Table K.3: DC, Table K.5: AC), the canonical
 * code assignment of Annex C, byte stuffing (a 0x00 after every 0xFF,
 * F.1.2.3) and padding of the last byte with 1-bits.
 * ------------------------------------------------------------------- */
static const uint8_t K3_BITS[16] = {0, 1, 5, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0, 0, 0};
static const uint8_t K3_VALS[12] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11};
static const uint8_t K5_BITS[16] = {0, 2, 1, 3, 3, 2, 4, 3, 5, 5, 4, 4, 0, 0, 1, 125};
static const uint8_t K5_VALS[162] = {
    0x01, 0x02, 0x03, 0x00, 0x04, 0x11, 0x05, 0x12, 0x21, 0x31, 0x41, 0x06, 0x13, 0x51, 0x61, 0x07,
    0x22, 0x71, 0x14, 0x32, 0x81, 0x91, 0xa1, 0x08, 0x23, 0x42, 0xb1, 0xc1, 0x15, 0x52, 0xd1, 0xf0,
    0x24, 0x33, 0x62, 0x72, 0x82, 0x09, 0x0a, 0x16, 0x17, 0x18, 0x19, 0x1a, 0x25, 0x26, 0x27, 0x28,
    0x29, 0x2a, 0x34, 0x35, 0x36, 0x37, 0x38, 0x39, 0x3a, 0x43, 0x44, 0x45, 0x46, 0x47, 0x48, 0x49,
    0x4a, 0x53, 0x54, 0x55, 0x56, 0x57, 0x58, 0x59, 0x5a, 0x63, 0x64, 0x65, 0x66, 0x67, 0x68, 0x69,
    0x6a, 0x73, 0x74, 0x75, 0x76, 0x77, 0x78, 0x79, 0x7a, 0x83, 0x84, 0x85, 0x86, 0x87, 0x88, 0x89,
    0x8a, 0x92, 0x93, 0x94, 0x95, 0x96, 0x97, 0x98, 0x99, 0x9a, 0xa2, 0xa3, 0xa4, 0xa5, 0xa6, 0xa7,
    0xa8, 0xa9, 0xaa, 0xb2, 0xb3, 0xb4, 0xb5, 0xb6, 0xb7, 0xb8, 0xb9, 0xba, 0xc2, 0xc3, 0xc4, 0xc5,
    0xc6, 0xc7, 0xc8, 0xc9, 0xca, 0xd2, 0xd3, 0xd4, 0xd5, 0xd6, 0xd7, 0xd8, 0xd9, 0xda, 0xe1, 0xe2,
    0xe3, 0xe4, 0xe5, 0xe6, 0xe7, 0xe8, 0xe9, 0xea, 0xf1, 0xf2, 0xf3, 0xf4, 0xf5, 0xf6, 0xf7, 0xf8,
    0xf9, 0xfa};

typedef struct {
    uint16_t code[256];
    uint8_t len[256]; /* 0: no code for this symbol */
} huff_table;

/* Annex C: codes of each length are consecutive; the first code of length
 * l + 1 is (the code after the last one of length l) shifted left by one */
static void huff_build(const uint8_t* bits, const uint8_t* vals, huff_table* t) {
    memset(t, 0, sizeof(*t));
    uint32_t code = 0;
    int k = 0;
    for (int l = 1; l <= 16; ++l) {
        for (int i = 0; i < bits[l - 1]; ++i, ++k) {
            t->code[vals[k]] = (uint16_t)code++;
            t->len[vals[k]] = (uint8_t)l;
        }
        code <<= 1;
    }
}

void orc_huff_code(int ac, int symbol, int32_t* code, int32_t* len) {
    huff_table t;
    if (ac) huff_build(K5_BITS, K5_VALS, &t);
    else huff_build(K3_BITS, K3_VALS, &t);
    *code = t.code[symbol & 255];
    *len = t.len[symbol & 255];
}

/* zig-zag position k -> natural index (row * 8 + column): the anti-diagonals
 * i + j = d in turn, downwards on odd d, upwards on even d (Figure A.6) */
void orc_zigzag(int32_t* zz) {
    int k = 0;
    for (int d = 0; d < 15; ++d) {
        const int ilo = d < 8 ? 0 : d - 7, ihi = d < 8 ? d : 7;
        if (d & 1)
            for (int i = ilo; i <= ihi; ++i) zz[k++] = i * 8 + (d - i);
        else
            for (int i = ihi; i >= ilo; --i) zz[k++] = i * 8 + (d - i);
    }
}

typedef struct {
    uint8_t* out;
    int64_t n;
    uint32_t acc;
    int nacc;
} bit_writer;

static void put_bit(bit_writer* w, unsigned bit) {
    w->acc = (w->acc << 1) | (bit & 1u);
    if (++w->nacc == 8) {
        const uint8_t b = (uint8_t)w->acc;
        if (w->out) w->out[w->n] = b;
        w->n++;
        if (b == 0xFF) { /* byte stuffing */
            if (w->out) w->out[w->n] = 0x00;
            w->n++;
        }
        w->acc = 0;
        w->nacc = 0;
    }
}

static void put_bits(bit_writer* w, uint32_t v, int len) {
    for (int i = len - 1; i >= 0; --i) put_bit(w, (v >> i) & 1u);
}

/* magnitude category (Tables F.1 / F.2) and its extra bits (F.1.2.1.1) */
static int category(int v) {
    int a = v < 0 ? -v : v, s = 0;
    while (a) {
        ++s;
        a >>= 1;
    }
    return s;
}

static uint32_t extra_bits(int v, int s) {
    return (uint32_t)(v >= 0 ? v : v - 1) & ((1u << s) - 1u);
}

int64_t orc_jpeg_entropy(const int16_t* coefs, int64_t nblk, uint8_t* out) {
    huff_table dc, ac;
    huff_build(K3_BITS, K3_VALS, &dc);
    huff_build(K5_BITS, K5_VALS, &ac);
    int32_t zz[64];
    orc_zigzag(zz);
    bit_writer w = {out, 0, 0, 0};
    int pred = 0;
    for (int64_t b = 0; b < nblk; ++b) {
        const int16_t* c = coefs + b * 64;
        const int diff = c[0] - pred;
        pred = c[0];
        const int sd = category(diff);
        if (sd > 11) return -1;
        put_bits(&w, dc.code[sd], dc.len[sd]);
        put_bits(&w, extra_bits(diff, sd), sd);
        int run = 0;
        for (int k = 1; k < 64; ++k) {
            const int v = c[zz[k]];
            if (v == 0) {
                ++run;
                continue;
            }
            while (run > 15) {
                put_bits(&w, ac.code[0xF0], ac.len[0xF0]);
                run -= 16;
            }
            const int sa = category(v);
            if (sa > 10) return -1;
            const int sym = (run << 4) | sa;
            put_bits(&w, ac.code[sym], ac.len[sym]);
            put_bits(&w, extra_bits(v, sa), sa);
            run = 0;
        }
        if (run > 0) put_bits(&w, ac.code[0x00], ac.len[0x00]); /* EOB */
    }
    while (w.nacc != 0) put_bit(&w, 1u); /* pad with 1-bits */
    return w.n;
}

/* decoder (Annex F.2.2), for the round-trip check: returns 0, or -1 on a
 * malformed stream */
typedef struct {
    const uint8_t* in;
    int64_t n, pos;
    uint32_t acc;
    int nacc;
} bit_reader;

static int get_bit(bit_reader* r) {
    if (r->nacc == 0) {
        if (r->pos >= r->n) return -1;
        const uint8_t b = r->in[r->pos++];
        if (b == 0xFF) {
            if (r->pos >= r->n || r->in[r->pos] != 0x00) return -1;
            r->pos++; /* the stuffed zero */
        }
        r->acc = b;
        r->nacc = 8;
    }
    r->nacc--;
    return (int)((r->acc >> r->nacc) & 1u);
}

static int decode_symbol(bit_reader* r, const huff_table* t) {
    uint32_t code = 0;
    for (int l = 1; l <= 16; ++l) {
        const int bit = get_bit(r);
        if (bit < 0) return -1;
        code = (code << 1) | (uint32_t)bit;
        for (int s = 0; s < 256; ++s)
            if (t->len[s] == l && t->code[s] == code) return s;
    }
    return -1;
}

static int receive_extend(bit_reader* r, int s, int* v) {
    uint32_t x = 0;
    for (int i = 0; i < s; ++i) {
        const int bit = get_bit(r);
        if (bit < 0) return -1;
        x = (x << 1) | (uint32_t)bit;
    }
    *v = (s == 0) ? 0 : ((x >> (s - 1)) ? (int)x : (int)x - (1 << s) + 1);
    return 0;
}

int orc_jpeg_entropy_decode(const uint8_t* in, int64_t nbytes, int64_t nblk, int16_t* coefs) {
    huff_table dc, ac;
    huff_build(K3_BITS, K3_VALS, &dc);
    huff_build(K5_BITS, K5_VALS, &ac);
    int32_t zz[64];
    orc_zigzag(zz);
    bit_reader r = {in, nbytes, 0, 0, 0};
    int pred = 0;
    for (int64_t b = 0; b < nblk; ++b) {
        int16_t* c = coefs + b * 64;
        memset(c, 0, sizeof(int16_t) * 64);
        const int sd = decode_symbol(&r, &dc);
        int diff;
        if (sd < 0 || receive_extend(&r, sd, &diff)) return -1;
        pred += diff;
        c[0] = (int16_t)pred;
        for (int k = 1; k < 64;) {
            const int sym = decode_symbol(&r, &ac);
            if (sym < 0) return -1;
            if (sym == 0x00) break; /* EOB */
            if (sym == 0xF0) {
                k += 16;
                continue;
            }
            k += sym >> 4;
            if (k > 63) return -1;
            int v;
            if (receive_extend(&r, sym & 15, &v)) return -1;
            c[zz[k++]] = (int16_t)v;
        }
    }
    return 0;
}

int64_t orc_jpeg(const float* v, int rows, int cols, int quality,
                 int16_t* coefs, float* lohi, float* deq) {
    int32_t qt[64];
    orc_jpeg_qtable(quality, qt);
    const long n = (long)rows * cols;
    float lo = v[0], hi = v[0];
    for (long i = 1; i < n; ++i) {
        if (v[i] < lo) lo = v[i];
        if (v[i] > hi) hi = v[i];
    }
    lohi[0] = lo;
    lohi[1] = hi;
    const long nblk = (long)(rows / 8) * (cols / 8);
    if (!(hi > lo)) { /* constant segment: sent exactly */
        for (long i = 0; i < n; ++i) deq[i] = lo;
        memset(coefs, 0, sizeof(int16_t) * nblk * 64);
        return 0;
    }
    /* the sample map is FP32 on both sides: the values are 32-bit images */
    const float rng = hi - lo;
    const float inv = 255.0f / rng;
    const float step = rng / 255.0f;
    int64_t nnz = 0;
    for (int bi = 0; bi < rows / 8; ++bi)
        for (int bj = 0; bj < cols / 8; ++bj) {
            const long blk = (long)bi * (cols / 8) + bj;
            double f[64], F[64], G[64], g[64];
            for (int i = 0; i < 8; ++i)
                for (int j = 0; j < 8; ++j) {
                    float x = v[(long)(bi * 8 + i) * cols + bj * 8 + j];
                    float t = (x - lo) * inv;
                    float r = roundf(t); /* half away from zero */
                    if (r < 0.0f) r = 0.0f;
                    if (r > 255.0f) r = 255.0f;
                    f[i * 8 + j] = (double)r - 128.0;
                }
            orc_dct8x8(f, F);
            for (int p = 0; p < 64; ++p) {
                double qv = round(F[p] / qt[p]);
                coefs[blk * 64 + p] = (int16_t)qv;
                nnz += (qv != 0.0);
                G[p] = qv * qt[p];
            }
            orc_idct8x8(G, g);
            for (int i = 0; i < 8; ++i)
                for (int j = 0; j < 8; ++j) {
                    double r = round(g[i * 8 + j] + 128.0);
                    if (r < 0.0) r = 0.0;
                    if (r > 255.0) r = 255.0;
                    float sv = (float)r;
                    long o = (long)(bi * 8 + i) * cols + bj * 8 + j;
                    deq[o] = (sv == 255.0f) ? hi : lo + sv * step;
                }
        }
    return nnz;
}

/* ------------------------------------------------------------------ */
/* message graph                                                       */
/* ------------------------------------------------------------------ */

void orc_relay_tables(int M, const int32_t* adj, int32_t* dist, int32_t* first) {
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * M);
    for (int s = 0; s < M; ++s) {
        int32_t* d = dist + (long)s * M;
        for (int m = 0; m < M; ++m) d[m] = -1;
        int head = 0, tail = 0;
        d[s] = 0;
        queue[tail++] = s;
        while (head < tail) {
            int x = queue[head++];
            for (int y = 0; y < M; ++y)
                if (adj[x * M + y] && d[y] < 0) {
                    d[y] = d[x] + 1;
                    queue[tail++] = y;
                }
        }
        for (int m = 0; m < M; ++m) {
            if (m == s || d[m] < 0) { first[(long)s * M + m] = (m == s) ? s : -1; continue; }
            int cur = m;
            while (d[cur] > 1) { /* step to the lowest-id neighbour one hop closer to s */
                int par = -1;
                for (int p = 0; p < M && par < 0; ++p)
                    if (adj[p * M + cur] && d[p] == d[cur] - 1) par = p;
                cur = par;
            }
            first[(long)s * M + m] = cur;
        }
    }
    free(queue);
}

/* ------------------------------------------------------------------ */
/* Algorithm 4 with quantized aggregation (Eq. 21-24)                  */
/* ------------------------------------------------------------------ */

typedef struct {
    int N, M, D, S;
    const int32_t* seg_row_ptr;
    const int32_t* dist;
    const int32_t* first;
    const int32_t* edge_q;
    const int32_t* home_q;
    const double* hist;
} view_ctx;

/* relay lag of segment s at node m: one hop per iteration, the first hop is
 * the exchange of the iteration itself */
static int relay_lag(const view_ctx* v, int s, int m) {
    return (s == m) ? 0 : v->dist[(long)s * v->M + m] - 1;
}

/* quantizer of the message that carries segment s to node m */
static int msg_kind(const view_ctx* v, int s, int m) {
    if (s == m) return v->home_q[m];
    int f = v->first[(long)s * v->M + m];
    return v->edge_q[s * v->M + f];
}

/* node m's copy of x after k completed iterations: segment s holds the
 * message produced at iteration k - max(dist(s,m) - 1, 0) (one relay hop per
 * iteration), or, when `held` is given, the version held[s*M+m] that node m
 * last received (messages can be lost); version 0 is the initial zero */
static void build_view(const view_ctx* v, int slice, int m, int k, const int32_t* held, double* out) {
    const long n = (long)v->N * v->N;
    for (int s = 0; s < v->M; ++s) {
        const long r0 = (long)v->seg_row_ptr[s] * v->N, r1 = (long)v->seg_row_ptr[s + 1] * v->N;
        int j = held ? held[(long)s * v->M + m] : k - relay_lag(v, s, m);
        if (j < 1) {
            for (long i = r0; i < r1; ++i) out[i] = 0.0;
            continue;
        }
        const double* src = v->hist + (((long)(j % v->D) * 3 + msg_kind(v, s, m)) * v->S + slice) * n;
        for (long i = r0; i < r1; ++i) out[i] = src[i];
    }
}

/* Algorithm 1 (CTR, Eq. 5): E gradient steps u <- u - eta P^T (P u - d) over
 * every angle, from the u given (the paper starts from zero), for `batch`
 * independent slices. u [batch][N][N] in place; sino [batch][A][B]. */
void orc_ctr(int N, int B, int A, const double* c, const double* s, int batch, const double* sino,
             double eta, int E, double* u) {
    const long n = (long)N * N;
    int32_t* all = (int32_t*)malloc(sizeof(int32_t) * (A > 0 ? A : 1));
    for (int a = 0; a < A; ++a) all[a] = a;
    double* r = (double*)malloc(sizeof(double) * (long)A * B);
    double* g = (double*)malloc(sizeof(double) * n);
    for (int k = 0; k < batch; ++k) {
        double* uk = u + (long)k * n;
        const double* dk = sino + (long)k * A * B;
        for (int e = 0; e < E; ++e) {
            orc_project(N, B, c, s, A, all, 1, uk, r); /* P u */
            for (long i = 0; i < (long)A * B; ++i) r[i] -= dk[i]; /* - d */
            orc_backproject(N, B, c, s, A, all, 1, r, g); /* Delta_u = P^T (P u - d) */
            for (long i = 0; i < n; ++i) uk[i] -= eta * g[i];
        }
    }
    free(all);
    free(r);
    free(g);
}

/* Algorithm 2 for one node: E1 gradient steps u <- u - eta1 Delta with
 * Delta = P_m^T (P_m u - d_m) + rho (u - (x_m - lambda_m / rho)), the node's
 * view x_m and dual lambda_m held fixed (warm start from the u given).
 * d_sl [A][B] is the slice's whole sinogram (rows ang[0..na) are d_m);
 * r [na][B] and g [N][N] are scratch. Returns ||P_m u - d_m||^2 at the last
 * step (0 when E1 = 0). */
static double alg2_steps(int N, int B, const double* c, const double* s, int na, const int32_t* ang,
                         const double* d_sl, const double* xv, const double* lm, double rho,
                         double eta1, int E1, double* um, double* r, double* g) {
    const long n = (long)N * N;
    double resid2 = 0.0;
    for (int e = 0; e < E1; ++e) {
        orc_project(N, B, c, s, na, ang, 1, um, r); /* P_m u_m */
        for (int q = 0; q < na; ++q)
            for (int b = 0; b < B; ++b)
                r[(long)q * B + b] -= d_sl[(long)ang[q] * B + b]; /* - d_m */
        if (e == E1 - 1)
            for (long i = 0; i < (long)na * B; ++i) resid2 += r[i] * r[i];
        orc_backproject(N, B, c, s, na, ang, 1, r, g); /* P_m^T (P_m u_m - d_m) */
        for (long i = 0; i < n; ++i) {
            double delta = g[i] + rho * (um[i] - (xv[i] - lm[i] / rho));
            um[i] -= eta1 * delta;
        }
    }
    return resid2;
}

double orc_alg2_node(int N, int B, const double* c, const double* s, int na, const int32_t* ang,
                     const double* sino_slice, const double* xview, const double* lam, double rho,
                     double eta1, int E1, double* u) {
    double* r = (double*)malloc(sizeof(double) * (na > 0 ? (long)na * B : 1));
    double* g = (double*)malloc(sizeof(double) * (long)N * N);
    const double res = alg2_steps(N, B, c, s, na, ang, sino_slice, xview, lam, rho, eta1, E1, u, r, g);
    free(r);
    free(g);
    return res;
}

int orc_dadmm_iterate(int N, int B, int A, int S, int M,
                      const double* c, const double* s,
                      const int32_t* node_ang_ptr, const int32_t* node_ang,
                      const int32_t* seg_row_ptr,
                      const int32_t* adj, const int32_t* edge_q,
                      const int32_t* home_q,
                      double rho, const double* eta1, double eta2, int E1, int E2,
                      int km_k, int km_iters, int jpeg_quality, uint64_t seed,
                      int D, const double* sino, double* u, double* lam,
                      double* xseg, double* hist, int32_t* iter, double* stats,
                      const uint8_t* drop, int32_t* held, const double* msg_in) {
    const long n = (long)N * N;
    if (N <= 0 || B <= 0 || M <= 0 || S <= 0 || D <= 0 || km_k > 256) return -1;
    if (seg_row_ptr[0] != 0 || seg_row_ptr[M] != N) return -1;

    int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * M * M);
    int32_t* first = (int32_t*)malloc(sizeof(int32_t) * M * M);
    orc_relay_tables(M, adj, dist, first);
    int max_lag = 0;
    for (long i = 0; i < (long)M * M; ++i) {
        if (dist[i] < 0) { free(dist); free(first); return -2; } /* disconnected */
        if (dist[i] - 1 > max_lag) max_lag = dist[i] - 1;
    }
    /* the ring must still hold node 0's previous view for the change statistic */
    if (D < max_lag + 2) { free(dist); free(first); return -3; }

    view_ctx vc = {N, M, D, S, seg_row_ptr, dist, first, edge_q, home_q, hist};
    const int k = *iter;
    /* message versions held after this iteration: every node receives the newest
     * version that has reached it (k + 1 - lag) unless drop[s*M+m] says that
     * message was lost, in which case it keeps the one it holds; its own
     * segment is never lost. Every version read must still be in the ring. */
    int32_t* held1 = NULL;
    if (held) {
        held1 = (int32_t*)malloc(sizeof(int32_t) * M * M);
        for (int s_ = 0; s_ < M; ++s_)
            for (int m = 0; m < M; ++m) {
                const long i = (long)s_ * M + m;
                const int newest = k + 1 - relay_lag(&vc, s_, m);
                const int lost = drop && s_ != m && drop[i];
                held1[i] = (!lost && newest >= 1) ? newest : held[i];
                const int ok_u = held[i] < 1 || held[i] >= k + 1 - D;                    /* read by Alg. 2 */
                const int ok_d = held1[i] < 1 || held1[i] >= k + 2 - D;                  /* read by Eq. 24 */
                const int ok_c = m != 0 || held[i] < 1 || held[i] >= k + 2 - D;          /* change statistic */
                if (!(ok_u && ok_d && ok_c)) { free(held1); free(dist); free(first); return -4; }
            }
    }
    double* xv = (double*)malloc(sizeof(double) * n);
    double* xv0 = (double*)malloc(sizeof(double) * n);
    double* g = (double*)malloc(sizeof(double) * n);
    double* r = (double*)malloc(sizeof(double) * (long)A * B);
    float* seg32 = (float*)malloc(sizeof(float) * n);
    float* deq32 = (float*)malloc(sizeof(float) * n);
    uint8_t* codes = (uint8_t*)malloc((size_t)n);
    int16_t* coefs = (int16_t*)malloc(sizeof(int16_t) * n);
    float cent[256], lohi[2];

    for (int sl = 0; sl < S; ++sl) {
        double resid2 = 0.0, bytes = 0.0;
        const double* d_sl = sino + (long)sl * A * B;

        /* Algorithm 2 on every node: u_m <- u_m - eta1 Delta, E1 times */
        for (int m = 0; m < M; ++m) {
            double* um = u + ((long)sl * M + m) * n;
            const double* lm = lam + ((long)sl * M + m) * n;
            const int na = node_ang_ptr[m + 1] - node_ang_ptr[m];
            const int32_t* ang = node_ang + node_ang_ptr[m];
            build_view(&vc, sl, m, k, held, xv); /* x_m^k */
            resid2 += alg2_steps(N, B, c, s, na, ang, d_sl, xv, lm, rho, eta1[m], E1, um, r, g);
        }

        /* Algorithm 3 on every owner's segment, then its messages (Eq. 23) */
        const int slot = (k + 1) % D;
        for (int m = 0; m < M; ++m) {
            const double* um = u + ((long)sl * M + m) * n;
            const double* lm = lam + ((long)sl * M + m) * n;
            const long r0 = (long)seg_row_ptr[m] * N, r1 = (long)seg_row_ptr[m + 1] * N;
            double* xs = xseg + (long)sl * n;
            for (int e = 0; e < E2; ++e)
                for (long i = r0; i < r1; ++i) {
                    double delta = rho * (xs[i] - um[i] - lm[i] / rho);
                    xs[i] -= eta2 * delta;
                }
            int need[3] = {0, 0, 0};
            need[home_q[m]] = 1;
            for (int t = 0; t < M; ++t)
                if (t != m) need[msg_kind(&vc, m, t)] = 1;
            const long len = r1 - r0;
            const int rows = seg_row_ptr[m + 1] - seg_row_ptr[m];
            for (long i = 0; i < len; ++i) seg32[i] = (float)xs[r0 + i];
            double kind_bytes[3] = {4.0 * len, 0.0, 0.0};
            for (int q = 0; q < 3; ++q) {
                if (!need[q]) continue;
                double* dst = hist + (((long)slot * 3 + q) * S + sl) * n + r0;
                if (q == ORC_Q_NONE) {
                    for (long i = 0; i < len; ++i) dst[i] = xs[r0 + i];
                } else if (q == ORC_Q_KMEANS) {
                    uint64_t key = orc_kmeans_key(seed, sl, m, k + 1);
                    orc_kmeans(seg32, len, km_k, km_iters, key, codes, cent, deq32, NULL);
                    for (long i = 0; i < len; ++i) dst[i] = deq32[i];
                    int bits = 0;
                    while ((1 << bits) < km_k) ++bits;
                    kind_bytes[q] = bits * (double)len / 8.0 + 4.0 * km_k;
                } else {
                    orc_jpeg(seg32, rows, N, jpeg_quality, coefs, lohi, deq32);
                    for (long i = 0; i < len; ++i) dst[i] = deq32[i];
                    /* the entropy-coded blocks + (lo, hi); a constant segment is sent as lo alone */
                    const int64_t eb = (lohi[1] > lohi[0]) ? orc_jpeg_entropy(coefs, len / 64, NULL) : 0;
                    kind_bytes[q] = (double)eb + 8.0;
                }
                if (msg_in && q != ORC_Q_NONE) { /* the decisions supplied from outside */
                    const double* src = msg_in + ((long)q * S + sl) * n + r0;
                    for (long i = 0; i < len; ++i) dst[i] = src[i];
                }
            }
            for (int t = 0; t < M; ++t)
                if (t != m) bytes += kind_bytes[msg_kind(&vc, m, t)];
        }

        /* aggregation (Eq. 23) and dual update (Eq. 24) */
        double gap2 = 0.0, chg2 = 0.0, nrm2 = 0.0;
        for (int m = 0; m < M; ++m) {
            const double* um = u + ((long)sl * M + m) * n;
            double* lm = lam + ((long)sl * M + m) * n;
            build_view(&vc, sl, m, k + 1, held1, xv); /* x_m^{k+1} */
            if (m == 0) {
                build_view(&vc, sl, 0, k, held, xv0);
                for (long i = 0; i < n; ++i) {
                    chg2 += (xv[i] - xv0[i]) * (xv[i] - xv0[i]);
                    nrm2 += xv0[i] * xv0[i];
                }
            }
            for (long i = 0; i < n; ++i) {
                double pr = um[i] - xv[i];
                gap2 += pr * pr;
                lm[i] = lm[i] + rho * pr;
            }
        }
        double* st = stats + (long)sl * ORC_NSTAT;
        st[0] = gap2;
        st[1] = chg2;
        st[2] = nrm2;
        st[3] = resid2;
        st[4] = bytes;
    }
    *iter = k + 1;
    if (held) {
        memcpy(held, held1, sizeof(int32_t) * M * M);
        free(held1);
    }
    free(xv); free(xv0); free(g); free(r); free(seg32); free(deq32); free(codes); free(coefs);
    free(dist); free(first);
    return 0;
}


/* ---------------------------------------------------------------------
 * Neighbour-averaged consensus: the decentralized analogue of the standard
 * ADMM x-update (Eq. 9: x = mean over all nodes of u_m + lambda_m / rho).
 * Every node keeps its own consensus image x_m and averages, over its closed
 * neighbourhood (itself and its graph neighbours), the messages
 * Q(u_j^{k+1} + lambda_j^k / rho) it receives in this iteration's exchange:
 *   u_m^{k+1}  = Algorithm 2 with x_m^k (warm start from u_m^k)
 *   v_j        = u_j^{k+1} + lambda_j^k / rho, quantized by the edge's
 *                quantizer (home quantizer for the node's own term)
 *   x_m^{k+1}  = (1 / |N[m]|) sum_{j in N[m]} Q_{j->m}(v_j)
 *   lambda_m^{k+1} = lambda_m^k + rho (u_m^{k+1} - x_m^{k+1})
 * On a complete graph without quantization this is Eq. 8-10 exactly.
 * State: u, lam [S][M][N*N], x [S][M][N*N]; stats as orc_dadmm_iterate
 * (chg2 / nrm2 of node 0's x; bytes = every message sent to a neighbour).
 * ------------------------------------------------------------------- */
int orc_consensus_iterate(int N, int B, int A, int S, int M,
                          const double* c, const double* s,
                          const int32_t* node_ang_ptr, const int32_t* node_ang,
                          const int32_t* adj, const int32_t* edge_q, const int32_t* home_q,
                          double rho, const double* eta1, int E1,
                          int km_k, int km_iters, int jpeg_quality, uint64_t seed,
                          const double* sino, double* u, double* lam, double* x,
                          int32_t* iter, double* stats) {
    const long n = (long)N * N;
    if (N <= 0 || B <= 0 || M <= 0 || S <= 0 || km_k > 256) return -1;
    const int k = *iter;
    double* g = (double*)malloc(sizeof(double) * n);
    double* r = (double*)malloc(sizeof(double) * (long)A * B);
    double* msg = (double*)malloc(sizeof(double) * 3 * M * n); /* [kind][j][n] of one slice */
    double* xn = (double*)malloc(sizeof(double) * n);
    float* v32 = (float*)malloc(sizeof(float) * n);
    float* deq32 = (float*)malloc(sizeof(float) * n);
    uint8_t* codes = (uint8_t*)malloc((size_t)n);
    int16_t* coefs = (int16_t*)malloc(sizeof(int16_t) * n);
    float cent[256], lohi[2];
    int bits = 0;
    while ((1 << bits) < km_k) ++bits;

    for (int sl = 0; sl < S; ++sl) {
        double resid2 = 0.0, bytes = 0.0, gap2 = 0.0, chg2 = 0.0, nrm2 = 0.0;
        const double* d_sl = sino + (long)sl * A * B;
        /* Algorithm 2 on every node with its own x_m^k */
        for (int m = 0; m < M; ++m) {
            double* um = u + ((long)sl * M + m) * n;
            const double* lm = lam + ((long)sl * M + m) * n;
            const double* xm = x + ((long)sl * M + m) * n;
            const int na = node_ang_ptr[m + 1] - node_ang_ptr[m];
            const int32_t* ang = node_ang + node_ang_ptr[m];
            for (int e = 0; e < E1; ++e) {
                orc_project(N, B, c, s, na, ang, 1, um, r);
                for (int q = 0; q < na; ++q)
                    for (int b = 0; b < B; ++b) r[(long)q * B + b] -= d_sl[(long)ang[q] * B + b];
                if (e == E1 - 1)
                    for (long i = 0; i < (long)na * B; ++i) resid2 += r[i] * r[i];
                orc_backproject(N, B, c, s, na, ang, 1, r, g);
                for (long i = 0; i < n; ++i) {
                    const double delta = g[i] + rho * (um[i] - (xm[i] - lm[i] / rho));
                    um[i] -= eta1[m] * delta;
                }
            }
        }
        /* every node's message v_j in the quantizers it is sent with */
        for (int j = 0; j < M; ++j) {
            const double* uj = u + ((long)sl * M + j) * n;
            const double* lj = lam + ((long)sl * M + j) * n;
            double* v = msg + (0L * M + j) * n;
            for (long i = 0; i < n; ++i) v[i] = uj[i] + lj[i] / rho;
            int need[3] = {0, 0, 0};
            need[home_q[j]] = 1;
            for (int m = 0; m < M; ++m)
                if (m != j && adj[j * M + m]) need[edge_q[j * M + m]] = 1;
            for (long i = 0; i < n; ++i) v32[i] = (float)v[i];
            double kind_bytes[3] = {4.0 * n, 0.0, 0.0};
            if (need[ORC_Q_KMEANS]) {
                orc_kmeans(v32, n, km_k, km_iters, orc_kmeans_key(seed, sl, j, k + 1), codes, cent, deq32, NULL);
                for (long i = 0; i < n; ++i) msg[(1L * M + j) * n + i] = deq32[i];
                kind_bytes[1] = bits * (double)n / 8.0 + 4.0 * km_k;
            }
            if (need[ORC_Q_JPEG]) {
                orc_jpeg(v32, N, N, jpeg_quality, coefs, lohi, deq32);
                for (long i = 0; i < n; ++i) msg[(2L * M + j) * n + i] = deq32[i];
                const int64_t eb = (lohi[1] > lohi[0]) ? orc_jpeg_entropy(coefs, n / 64, NULL) : 0;
                kind_bytes[2] = (double)eb + 8.0;
            }
            for (int m = 0; m < M; ++m)
                if (m != j && adj[j * M + m]) bytes += kind_bytes[edge_q[j * M + m]];
        }
        /* neighbourhood averages and dual update */
        for (int m = 0; m < M; ++m) {
            double* xm = x + ((long)sl * M + m) * n;
            const double* um = u + ((long)sl * M + m) * n;
            double* lm = lam + ((long)sl * M + m) * n;
            int cnt = 1;
            const double* own = msg + ((long)home_q[m] * M + m) * n;
            for (long i = 0; i < n; ++i) xn[i] = own[i];
            for (int j = 0; j < M; ++j)
                if (j != m && adj[j * M + m]) {
                    const double* mj = msg + ((long)edge_q[j * M + m] * M + j) * n;
                    for (long i = 0; i < n; ++i) xn[i] += mj[i];
                    ++cnt;
                }
            for (long i = 0; i < n; ++i) xn[i] /= cnt;
            if (m == 0)
                for (long i = 0; i < n; ++i) {
                    chg2 += (xn[i] - xm[i]) * (xn[i] - xm[i]);
                    nrm2 += xm[i] * xm[i];
                }
            for (long i = 0; i < n; ++i) {
                xm[i] = xn[i];
                const double pr = um[i] - xm[i];
                gap2 += pr * pr;
                lm[i] += rho * pr;
            }
        }
        double* st = stats + (long)sl * ORC_NSTAT;
        st[0] = gap2;
        st[1] = chg2;
        st[2] = nrm2;
        st[3] = resid2;
        st[4] = bytes;
    }
    *iter = k + 1;
    free(g); free(r); free(msg); free(xn); free(v32); free(deq32); free(codes); free(coefs);
    return 0;
}
