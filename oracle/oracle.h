/*
 * Plain FP64 CPU oracle for decentralized ADMM tomography with quantized
 * messages ("Distributed Tomographic Reconstruction with Quantization",
 * arXiv 2410.06106).
 *
 * THIS IS TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it. The CUDA library never links,
 * includes or calls anything here, and nothing here includes the CUDA
 * library's headers.
 *
 * Geometry convention (the paper leaves it open, Sec. 2.1):
 *   pixel (i, j) of an N x N image is the unit square centred at
 *     x_j = j - (N-1)/2,  y_i = (N-1)/2 - i    (row 0 at the top, y up);
 *   ray (a, b) is the line  x cos(theta_a) + y sin(theta_a) = t_b,
 *     t_b = b - (B-1)/2,  unit detector spacing;
 *   P[(a,b),(i,j)] = length of the intersection of that line with that
 *     pixel (Eq. 2). A line lying exactly on the common edge of two pixels
 *     gives each of them half of the edge length.
 *
 * All image / sinogram arrays are row-major and contiguous.
 */
#ifndef TOMO_ORACLE_H
#define TOMO_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* number of OpenMP threads the oracle runs with */
int orc_num_threads(void);

/* threads of the oracle's parallel loops from now on (results do not depend on it) */
void orc_set_num_threads(int n);

/* cos/sin of each angle; multiples of pi/2 (within 1e-12 rad) are snapped to
 * exact 0 / +-1. */
void orc_trig(int n, const double* theta, double* c, double* s);

/* Eq. 2 entry: length of the line {x c + y s = t} inside the unit square
 * centred at (xc, yc), by clipping the line against the square. */
double orc_chord(double c, double s, double t, double xc, double yc);

/* Eq. 4, d = P u, for the angle rows aidx[0..nsel).
 * img [batch][N][N], sino [batch][nsel][B]. */
void orc_project(int N, int B, const double* c, const double* s, int nsel,
                 const int32_t* aidx, int batch, const double* img, double* sino);

/* transpose: img = P^T sino, same layouts */
void orc_backproject(int N, int B, const double* c, const double* s, int nsel,
                     const int32_t* aidx, int batch, const double* sino, double* img);

/* single rays (ray_a[r], ray_b[r]) of P u; img [N][N] */
void orc_project_rays(int N, int B, const double* c, const double* s, int nray,
                      const int32_t* ray_a, const int32_t* ray_b,
                      const double* img, double* out);

/* single pixels pix[q] (flat index i*N+j) of P^T sino; sino [nsel][B] */
void orc_backproject_pixels(int N, int B, const double* c, const double* s,
                            int nsel, const int32_t* aidx, const double* sino,
                            int npix, const int32_t* pix, double* out);

/* Algorithm 1 (centralized reconstruction, Eq. 5): E steps of
 *   u <- u - eta P^T (P u - d)
 * over every angle, from the u given, in place; `batch` slices:
 * u [batch][N][N], sino [batch][A][B]. */
void orc_ctr(int N, int B, int A, const double* c, const double* s, int batch, const double* sino,
             double eta, int E, double* u);

/* Algorithm 2 for a single node m: E1 steps of
 *   u <- u - eta1 (P_m^T (P_m u - d_m) + rho (u - (x_m - lambda_m / rho)))
 * from the u given (in place), with the node's view x_m (xview) and dual
 * lambda_m (lam) held fixed. ang[0..na) are the node's angle indices,
 * sino_slice [A][B] the slice's sinogram (rows ang[q] are d_m). All images
 * [N][N]. Returns ||P_m u - d_m||^2 at the last step (0 if E1 = 0). */
double orc_alg2_node(int N, int B, const double* c, const double* s, int na, const int32_t* ang,
                     const double* sino_slice, const double* xview, const double* lam, double rho,
                     double eta1, int E1, double* u);

/* ||P_sel||_2^2 by power iteration on P^T P from a seeded start vector */
double orc_opnorm_sq(int N, int B, const double* c, const double* s, int nsel,
                     const int32_t* aidx, int iters, uint64_t seed);

/* splitmix64 output function (Steele, Lea & Flood 2014) and the counter key
 * used for K-means initialisation of owner `owner`, slice `slice` at ADMM
 * iteration `iter`. */
uint64_t orc_mix64(uint64_t z);
uint64_t orc_kmeans_key(uint64_t seed, int slice, int owner, int iter);

/* Algorithm 5: scalar K-means quantizer of v[0..n). codes [n], cent [k],
 * deq [n]; obj [iters+1] (nullable) receives the distortion after every
 * assignment step. */
void orc_kmeans(const float* v, int64_t n, int k, int iters, uint64_t key,
                uint8_t* codes, float* cent, float* deq, double* obj);

/* JPEG luminance table scaled to `quality` (IJG rule), natural order */
void orc_jpeg_qtable(int quality, int32_t* qt);

/* orthonormal 8x8 DCT-II and its inverse, FP64, natural order */
void orc_dct8x8(const double* in, double* out);
void orc_idct8x8(const double* in, double* out);

/* JPEG-style codec of a rows x cols segment (both multiples of 8).
 * coefs [rows/8][cols/8][64], lohi [2], deq [rows][cols].
 * Returns the number of non-zero quantized coefficients. */
int64_t orc_jpeg(const float* v, int rows, int cols, int quality,
                 int16_t* coefs, float* lohi, float* deq);

/* Baseline Huffman entropy coding of quantized blocks (ITU-T T.81 Annex
 * F.1.2 with the luminance tables K.3 / K.5): coefs [nblk][64] in natural
 * order, blocks in raster order (one DC predictor over the whole array).
 * Returns the length in bytes of the entropy-coded segment (stuffed, padded
 * with 1-bits), -1 if a coefficient is out of the baseline range; writes the
 * bytes to out unless it is NULL. */
int64_t orc_jpeg_entropy(const int16_t* coefs, int64_t nblk, uint8_t* out);
int orc_jpeg_entropy_decode(const uint8_t* in, int64_t nbytes, int64_t nblk, int16_t* coefs);
/* code word and length of a DC category (ac = 0) or AC run/size symbol (ac = 1) */
void orc_huff_code(int ac, int symbol, int32_t* code, int32_t* len);
/* zig-zag position -> natural index (Figure A.6) */
void orc_zigzag(int32_t* zz);

/* Relay tables of the message graph: dist[s*M+m] = hop distance from owner s
 * to node m (-1 if unreachable), first[s*M+m] = the neighbour of s on the
 * shortest path to m that always takes the lowest-id parent. */
void orc_relay_tables(int M, const int32_t* adj, int32_t* dist, int32_t* first);

/* quantizer kinds */
#define ORC_Q_NONE   0
#define ORC_Q_KMEANS 1
#define ORC_Q_JPEG   2

/* per-slice statistics written by orc_dadmm_iterate */
#define ORC_NSTAT 5   /* gap2, change2, norm2_prev, resid2, bytes */

/* One dADMM iteration (Algorithm 4 with Algorithms 2, 3 and Eq. 21-24) for
 * S independent slices of M nodes each. See oracle.c for the step list.
 * Lost messages: held [M][M] (NULL: none are lost) is the version of owner
 * s's segment that node m holds (held[s*M+m], 0 = none yet), read for x_m^k
 * and updated to x_m^{k+1}; drop [M][M] (NULL: none lost this iteration)
 * marks the messages lost in this iteration's exchange, for every slice.
 *   sino  [S][A][B]          measured data, natural angle order
 *   u,lam [S][M][N*N]        local images and duals (updated)
 *   xseg  [S][N*N]           every owner's unquantized segment (updated)
 *   hist  [D][3][S][N*N]     dequantized messages, ring of depth
 *                            D >= max(hop distance) + 1
 *   iter  in: completed iterations k; out: k+1
 *   stats [S][ORC_NSTAT]
 *   msg_in [3][S][N*N] or NULL: dequantized messages to use in place of the
 *                            quantizers' output (planes ORC_Q_KMEANS and
 *                            ORC_Q_JPEG; the identity plane is always the
 *                            owner's own segment): Algorithm 4 with its
 *                            discrete decisions supplied from outside, which
 *                            separates the continuous arithmetic from the
 *                            quantizers' decisions when two implementations
 *                            are compared; bytes are still counted from the
 *                            oracle's own quantizers
 * Returns 0, a negative code for invalid arguments, or -4 when a held
 * version has left the message ring (depth D). */
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
                      const uint8_t* drop, int32_t* held, const double* msg_in);

/* Neighbour-averaged consensus (the decentralized analogue of Eq. 9; see
 * oracle.c): x [S][M][N*N] is every node's own consensus image; messages are
 * full images u_j + lambda_j / rho quantized per edge. */
int orc_consensus_iterate(int N, int B, int A, int S, int M,
                          const double* c, const double* s,
                          const int32_t* node_ang_ptr, const int32_t* node_ang,
                          const int32_t* adj, const int32_t* edge_q, const int32_t* home_q,
                          double rho, const double* eta1, int E1,
                          int km_k, int km_iters, int jpeg_quality, uint64_t seed,
                          const double* sino, double* u, double* lam, double* x,
                          int32_t* iter, double* stats);

#ifdef __cplusplus
}
#endif
#endif
