/*
 * drt3d_oracle.c -- plain, slow CPU oracle for the 3D multiscale discrete
 * Radon transform (DRT) of planes and the discrete John transform (DJT) of
 * lines of Marichal-Hernandez et al., "Three-dimensional multiscale discrete
 * Radon and John transforms" (arXiv 2501.13664).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * GPU library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library, and it is never on the
 * product path.
 *
 * Conventions (all arrays C-contiguous, caller-owned):
 *   - N = 2^n, 2 <= N <= 1024.
 *   - a volume in one dodecant/sector frame is g[x][y][z], N^3 values;
 *   - planes output of one dodecant:  R[s1][s2][d], d in [0, 3N), the storage
 *     index of Algorithm 1 (the volume is embedded at d in [2N, 3N)), so the
 *     plane is z = l_{s1}(x) + l_{s2}(y) + d - 2N;
 *   - lines output of one sector: J[s1][s2][d1][d2], d1, d2 in [0, 2N), the
 *     storage index of Algorithm 3 (volume embedded at [N, 2N) on both), so
 *     the line is y = l_{s1}(x) + d1 - N, z = l_{s2}(x) + d2 - N.
 *   - int32 arithmetic wraps modulo 2^32 (computed in uint32_t).
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int ilog2(int N) {
    int n = 0;
    while ((1 << n) < N) ++n;
    return n;
}

/* ------------------------------------------------------------------------ */
/* Digital line, eq.(digitalLine) (Section 2.1).                             */
/*   l^n_s(u) = sum_{i=0}^{n-1} u_{n-1-i} * floor((floor(s/2^i) + 1) / 2)    */
/* with u_j the j-th bit of u (lambda(u) = sum u_j 2^j).  For non-negative    */
/* integers floor(s/2^i) is s >> i.                                           */
/* ------------------------------------------------------------------------ */
int64_t drto_lline(int n, int64_t s, int64_t u) {
    int64_t acc = 0;
    for (int i = 0; i < n; ++i) {
        int64_t bit = (u >> (n - 1 - i)) & 1;
        acc += bit * (((s >> i) + 1) >> 1);
    }
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Dodecant input maps (Algorithm 2, InOrder).  The printed table covers     */
/* only 10 distinct normal sectors; the reading used here flips original     */
/* axis j where entry j is negative, then takes new axis i from original     */
/* axis |entry i|, with single-sign fixes on rows 5, 6, 9 and 10.  Dodecant  */
/* k's frame volume is g_k(x', y', z') = f(index returned below).            */
/* Returns the flat index x*N*N + y*N + z into f.                            */
/* ------------------------------------------------------------------------ */
int64_t drto_dodecant_src(int N, int k, int xp, int yp, int zp) {
    const int M = N - 1;
    int x, y, z;
    switch (k) {
    case 0:  x = xp;      y = yp;      z = zp;      break; /* [ 1, 2, 3] */
    case 1:  x = M - yp;  y = xp;      z = zp;      break; /* [-2, 1, 3] */
    case 2:  x = M - xp;  y = M - yp;  z = zp;      break; /* [-1,-2, 3] */
    case 3:  x = yp;      y = M - xp;  z = zp;      break; /* [ 2,-1, 3] */
    case 4:  x = M - xp;  y = M - zp;  z = M - yp;  break; /* [-1,-3,-2] */
    case 5:  x = M - yp;  y = zp;      z = xp;      break; /* [-3, 1, 2] */
    case 6:  x = yp;      y = M - zp;  z = xp;      break; /* [ 3,-1, 2] */
    case 7:  x = xp;      y = zp;      z = M - yp;  break; /* [ 1, 3,-2] */
    case 8:  x = M - zp;  y = M - yp;  z = M - xp;  break; /* [-3,-2,-1] */
    case 9:  x = zp;      y = M - xp;  z = yp;      break; /* [ 2,-3, 1] */
    case 10: x = M - zp;  y = xp;      z = yp;      break; /* [-2, 3, 1] */
    default: x = zp;      y = yp;      z = M - xp;  break; /* [ 3, 2,-1] */
    }
    return ((int64_t)x * N + y) * N + z;
}

/* DJT sectors (Section 4: twelve sets of lines, x-, y- and z-driven, four   */
/* each).  Sector k = 4*a + flips drives along axis a in (x, y, z); the two  */
/* other axes (b, c) follow in cyclic order, bit 0 of flips reverses b and   */
/* bit 1 reverses c.  Frame: x' along a, y' along b, z' along c.             */
int64_t drto_sector_src(int N, int k, int xp, int yp, int zp) {
    const int M = N - 1;
    int a = k >> 2, fl = k & 3;
    int yb = (fl & 1) ? M - yp : yp;
    int zc = (fl & 2) ? M - zp : zp;
    int c[3];
    /* axis a gets x', axis (a+1)%3 gets yb, axis (a+2)%3 gets zc */
    c[a] = xp;
    c[(a + 1) % 3] = yb;
    c[(a + 2) % 3] = zc;
    return ((int64_t)c[0] * N + c[1]) * N + c[2];
}

/* g[x'][y'][z'] = f[src(x',y',z')] for 4-byte elements (int32 or float). */
void drto_gather_dodecant_4(int N, int k, const uint32_t* f, uint32_t* g) {
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y)
            for (int z = 0; z < N; ++z)
                g[((int64_t)x * N + y) * N + z] = f[drto_dodecant_src(N, k, x, y, z)];
}
void drto_gather_dodecant_8(int N, int k, const uint64_t* f, uint64_t* g) {
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y)
            for (int z = 0; z < N; ++z)
                g[((int64_t)x * N + y) * N + z] = f[drto_dodecant_src(N, k, x, y, z)];
}
/* Adjoint of the gather: f[src(x',y',z')] += g[x'][y'][z'] (double). */
void drto_scatter_add_dodecant_f64(int N, int k, const double* g, double* f) {
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y)
            for (int z = 0; z < N; ++z)
                f[drto_dodecant_src(N, k, x, y, z)] += g[((int64_t)x * N + y) * N + z];
}
void drto_scatter_add_dodecant_i32(int N, int k, const int32_t* g, int32_t* f) {
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y)
            for (int z = 0; z < N; ++z) {
                int64_t s = drto_dodecant_src(N, k, x, y, z);
                f[s] = (int32_t)((uint32_t)f[s] + (uint32_t)g[((int64_t)x * N + y) * N + z]);
            }
}
/* idx[x'][y'][z'] = flat index into f of g_k(x', y', z'). */
void drto_dodecant_index_table(int N, int k, int64_t* idx) {
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y)
            for (int z = 0; z < N; ++z)
                idx[((int64_t)x * N + y) * N + z] = drto_dodecant_src(N, k, x, y, z);
}
void drto_sector_index_table(int N, int k, int64_t* idx) {
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y)
            for (int z = 0; z < N; ++z)
                idx[((int64_t)x * N + y) * N + z] = drto_sector_src(N, k, x, y, z);
}
void drto_gather_sector_4(int N, int k, const uint32_t* f, uint32_t* g) {
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y)
            for (int z = 0; z < N; ++z)
                g[((int64_t)x * N + y) * N + z] = f[drto_sector_src(N, k, x, y, z)];
}

/* ------------------------------------------------------------------------ */
/* Planes, definition eq.(3DfDRT): brute-force scatter of every voxel onto   */
/* the one displacement it lies on for each slope pair.                      */
/*   R[s1][s2][d] = sum_{x,y} g(x, y, l_{s1}(x) + l_{s2}(y) + d - 2N)        */
/* Accumulates in int64 (exact for any int32 input) or double.               */
/* ------------------------------------------------------------------------ */
void drto_planes_brute_i64(int N, const int64_t* g, int64_t* R) {
    const int n = ilog2(N), W = 3 * N;
    memset(R, 0, sizeof(int64_t) * (size_t)N * N * W);
    for (int s1 = 0; s1 < N; ++s1)
        for (int s2 = 0; s2 < N; ++s2)
            for (int x = 0; x < N; ++x) {
                const int64_t l1 = drto_lline(n, s1, x);
                for (int y = 0; y < N; ++y) {
                    const int64_t l2 = drto_lline(n, s2, y);
                    for (int z = 0; z < N; ++z) {
                        const int64_t d = z - l1 - l2 + 2 * N;
                        R[((int64_t)s1 * N + s2) * W + d] += g[((int64_t)x * N + y) * N + z];
                    }
                }
            }
}
void drto_planes_brute_f64(int N, const double* g, double* R) {
    const int n = ilog2(N), W = 3 * N;
    memset(R, 0, sizeof(double) * (size_t)N * N * W);
    for (int s1 = 0; s1 < N; ++s1)
        for (int s2 = 0; s2 < N; ++s2)
            for (int x = 0; x < N; ++x) {
                const int64_t l1 = drto_lline(n, s1, x);
                for (int y = 0; y < N; ++y) {
                    const int64_t l2 = drto_lline(n, s2, y);
                    for (int z = 0; z < N; ++z) {
                        const int64_t d = z - l1 - l2 + 2 * N;
                        R[((int64_t)s1 * N + s2) * W + d] += g[((int64_t)x * N + y) * N + z];
                    }
                }
            }
}
/* One cell of eq.(3DfDRT) in its gather form, int64: O(N^2). */
int64_t drto_planes_cell_i64(int N, const int32_t* g, int s1, int s2, int d) {
    const int n = ilog2(N);
    int64_t acc = 0;
    for (int x = 0; x < N; ++x) {
        const int64_t l1 = drto_lline(n, s1, x);
        for (int y = 0; y < N; ++y) {
            const int64_t z = l1 + drto_lline(n, s2, y) + d - 2 * N;
            if (z >= 0 && z < N) acc += g[((int64_t)x * N + y) * N + z];
        }
    }
    return acc;
}
/* Transpose of the brute force: gbar[x][y][z] = sum_{s1,s2} Rbar[s1][s2][d(x,y,z)]. */
void drto_planes_adjoint_brute_f64(int N, const double* Rbar, double* gbar) {
    const int n = ilog2(N), W = 3 * N;
    memset(gbar, 0, sizeof(double) * (size_t)N * N * N);
    for (int s1 = 0; s1 < N; ++s1)
        for (int s2 = 0; s2 < N; ++s2)
            for (int x = 0; x < N; ++x) {
                const int64_t l1 = drto_lline(n, s1, x);
                for (int y = 0; y < N; ++y) {
                    const int64_t l2 = drto_lline(n, s2, y);
                    for (int z = 0; z < N; ++z) {
                        const int64_t d = z - l1 - l2 + 2 * N;
                        gbar[((int64_t)x * N + y) * N + z] += Rbar[((int64_t)s1 * N + s2) * W + d];
                    }
                }
            }
}

/* ------------------------------------------------------------------------ */
/* Planes, Algorithm 1 (basicDRT3D) with the stage map eq.(map3D).           */
/* Two N x N x 3N buffers; the volume is placed at d in [2N, 3N); reads at   */
/* d >= 3N are 0; n stages, each writing one datum from four reads.  The     */
/* iterations of one stage are independent, so the d loop is run innermost   */
/* (memory order) instead of outermost; the values are the same.             */
/* ------------------------------------------------------------------------ */
#define DRTO_ALG1_BODY(T)                                                            \
    const int n = ilog2(N), W = 3 * N;                                              \
    const size_t cells = (size_t)N * N * W;                                         \
    T* fm = (T*)calloc(cells, sizeof(T));                                           \
    T* fn = (T*)calloc(cells, sizeof(T));                                           \
    if (!fm || !fn) { free(fm); free(fn); return -1; }                              \
    for (int x = 0; x < N; ++x)                                                     \
        for (int y = 0; y < N; ++y)                                                 \
            for (int z = 0; z < N; ++z)                                             \
                fm[((size_t)x * N + y) * W + 2 * N + z] = (T)g[((size_t)x * N + y) * N + z]; \
    for (int m = 0; m < n; ++m) {                                                   \
        const int V = 1 << (n - m - 1), S = 1 << m;                                 \
        for (int v1 = 0; v1 < V; ++v1)                                              \
        for (int sg1 = 0; sg1 < S; ++sg1)                                           \
        for (int v2 = 0; v2 < V; ++v2)                                              \
        for (int sg2 = 0; sg2 < S; ++sg2)                                           \
        for (int l1 = 0; l1 < 2; ++l1)                                              \
        for (int l2 = 0; l2 < 2; ++l2) {                                            \
            const int a1 = sg1 + (v1 << (m + 1)), b1 = a1 + S;                      \
            const int a2 = sg2 + (v2 << (m + 1)), b2 = a2 + S;                      \
            const int o1 = l1 + (sg1 << 1) + (v1 << (m + 1));                       \
            const int o2 = l2 + (sg2 << 1) + (v2 << (m + 1));                       \
            const int sh1 = sg1 + l1, sh2 = sg2 + l2;                               \
            const T* r00 = fm + ((size_t)a1 * N + a2) * W;                          \
            const T* r10 = fm + ((size_t)b1 * N + a2) * W;                          \
            const T* r01 = fm + ((size_t)a1 * N + b2) * W;                          \
            const T* r11 = fm + ((size_t)b1 * N + b2) * W;                          \
            T* out = fn + ((size_t)o1 * N + o2) * W;                                \
            for (int d = 0; d < W; ++d) {                                           \
                T f00 = r00[d];                                                     \
                T f10 = (d + sh1 < W) ? r10[d + sh1] : (T)0;                        \
                T f01 = (d + sh2 < W) ? r01[d + sh2] : (T)0;                        \
                T f11 = (d + sh1 + sh2 < W) ? r11[d + sh1 + sh2] : (T)0;            \
                out[d] = f00 + f10 + f01 + f11;                                     \
            }                                                                       \
        }                                                                           \
        T* t = fm; fm = fn; fn = t;                                                 \
    }                                                                               \
    memcpy(R, fm, cells * sizeof(T));                                               \
    free(fm); free(fn);                                                             \
    return 0;

int drto_planes_alg1_i32(int N, const int32_t* g, int32_t* R_) {
    uint32_t* R = (uint32_t*)R_;
    DRTO_ALG1_BODY(uint32_t)
}
int drto_planes_alg1_f64(int N, const double* g, double* R) {
    DRTO_ALG1_BODY(double)
}

/* ------------------------------------------------------------------------ */
/* Planes adjoint (backprojection), Section 5.1: the stage loop of           */
/* Algorithm 1 reversed, with eq.(invmap3Dsummation):                        */
/*   fb^m(s1|v1m,v1|s2|v2m,v2|d) = sum_{l1,l2} fb^{m+1}(l1,s1|v1|l2,s2|v2|    */
/*                 d - v1m (l1 + s1) - v2m (l2 + s2)),  reads at d < 0 are 0. */
/* The result is fb^0 restricted to d in [2N, 3N) (the embedding's adjoint). */
/* ------------------------------------------------------------------------ */
#define DRTO_ADJ_BODY(T)                                                             \
    const int n = ilog2(N), W = 3 * N;                                              \
    const size_t cells = (size_t)N * N * W;                                         \
    T* fm = (T*)malloc(cells * sizeof(T));                                          \
    T* fn = (T*)malloc(cells * sizeof(T));                                          \
    if (!fm || !fn) { free(fm); free(fn); return -1; }                              \
    memcpy(fn, Rbar, cells * sizeof(T));                                            \
    for (int m = n - 1; m >= 0; --m) {                                              \
        const int V = 1 << (n - m - 1), S = 1 << m;                                 \
        for (int v1 = 0; v1 < V; ++v1)                                              \
        for (int sg1 = 0; sg1 < S; ++sg1)                                           \
        for (int v1m = 0; v1m < 2; ++v1m)                                           \
        for (int v2 = 0; v2 < V; ++v2)                                              \
        for (int sg2 = 0; sg2 < S; ++sg2)                                           \
        for (int v2m = 0; v2m < 2; ++v2m) {                                         \
            const int i1 = sg1 + (v1m << m) + (v1 << (m + 1));                      \
            const int i2 = sg2 + (v2m << m) + (v2 << (m + 1));                      \
            T* out = fm + ((size_t)i1 * N + i2) * W;                                \
            for (int d = 0; d < W; ++d) out[d] = (T)0;                              \
            for (int l1 = 0; l1 < 2; ++l1)                                          \
            for (int l2 = 0; l2 < 2; ++l2) {                                        \
                const int o1 = l1 + (sg1 << 1) + (v1 << (m + 1));                   \
                const int o2 = l2 + (sg2 << 1) + (v2 << (m + 1));                   \
                const int sh = v1m * (l1 + sg1) + v2m * (l2 + sg2);                 \
                const T* src = fn + ((size_t)o1 * N + o2) * W;                      \
                for (int d = sh; d < W; ++d) out[d] += src[d - sh];                 \
            }                                                                       \
        }                                                                           \
        T* t = fm; fm = fn; fn = t;                                                 \
    }                                                                               \
    for (int x = 0; x < N; ++x)                                                     \
        for (int y = 0; y < N; ++y)                                                 \
            for (int z = 0; z < N; ++z)                                             \
                gbar[((size_t)x * N + y) * N + z] = fn[((size_t)x * N + y) * W + 2 * N + z]; \
    free(fm); free(fn);                                                             \
    return 0;

int drto_planes_adjoint_i32(int N, const int32_t* Rbar_, int32_t* gbar_) {
    const uint32_t* Rbar = (const uint32_t*)Rbar_;
    uint32_t* gbar = (uint32_t*)gbar_;
    DRTO_ADJ_BODY(uint32_t)
}
int drto_planes_adjoint_f64(int N, const double* Rbar, double* gbar) {
    DRTO_ADJ_BODY(double)
}

/* ------------------------------------------------------------------------ */
/* Exact integer inverse of one dodecant (not printed in the paper; derived  */
/* from eq.(map2D)/eq.(map3D) and the zero embedding of Algorithm 1).        */
/*                                                                          */
/* A stage of eq.(map3D) equals a half-stage along s1 followed by a          */
/* half-stage along s2 (the four terms regroup exactly, including the zero   */
/* reads past 3N).  One half-stage with slope-so-far sg and new bit l maps   */
/* the pair (lo = position bit 0, hi = position bit 1) to                    */
/*     out_l[d] = lo[d] + hi[d + sg + l]          (hi[>= 3N] = 0).            */
/* So Delta = out_1 - out_0 satisfies Delta[d] = hi[d+sg+1] - hi[d+sg], and   */
/*     hi[e] = -sum_{i = e-sg}^{3N-1-sg} Delta[i]   (e >= sg; 0 below),      */
/*     lo[d] = out_0[d] - hi[d + sg].                                        */
/* Data in the range of the forward map has Delta[d] = 0 for d >= 3N - sg    */
/* and, after all stages, zeros outside d in [2N, 3N); both are checked.     */
/* Stages are undone from m = n-1 down to 0, s2 half first, then s1.          */
/* Arithmetic is modulo 2^32 throughout, so the inverse is exact even when   */
/* the forward sums wrapped.  Returns 0 on success, 1 if R is not in range,  */
/* -1 on allocation failure.                                                 */
/* ------------------------------------------------------------------------ */
static int drto_undo_half(uint32_t* lo, uint32_t* hi, const uint32_t* out0,
                          const uint32_t* out1, int W, int sg, uint32_t* scratch) {
    int bad = 0;
    /* S[i] = sum_{i' = i}^{W-1-sg} Delta[i'], S[i] = 0 for i > W-1-sg. */
    uint32_t* S = scratch;
    uint32_t run = 0;
    for (int i = W - 1; i >= 0; --i) {
        uint32_t delta = out1[i] - out0[i];
        if (i > W - 1 - sg) {
            if (delta != 0) bad = 1;
            S[i] = 0;
        } else {
            run += delta;
            S[i] = run;
        }
    }
    for (int e = 0; e < W; ++e) hi[e] = (e >= sg) ? (uint32_t)0 - S[e - sg] : 0u;
    for (int d = 0; d < W; ++d) lo[d] = out0[d] - ((d + sg < W) ? hi[d + sg] : 0u);
    return bad;
}

int drto_planes_inverse_i32(int N, const int32_t* R_, int32_t* g_) {
    const uint32_t* R = (const uint32_t*)R_;
    uint32_t* g = (uint32_t*)g_;
    const int n = ilog2(N), W = 3 * N;
    const size_t cells = (size_t)N * N * W;
    uint32_t* fa = (uint32_t*)malloc(cells * sizeof(uint32_t));
    uint32_t* fb = (uint32_t*)malloc(cells * sizeof(uint32_t));
    uint32_t* scratch = (uint32_t*)malloc((size_t)W * sizeof(uint32_t));
    if (!fa || !fb || !scratch) { free(fa); free(fb); free(scratch); return -1; }
    memcpy(fa, R, cells * sizeof(uint32_t));
    int bad = 0;
    for (int m = n - 1; m >= 0; --m) {
        const int V = 1 << (n - m - 1), S = 1 << m;
        /* Undo the s2 half-stage: fa holds rows (o1 = s1 index at stage m+1,
           o2 = s2 index at stage m+1); fb receives (o1, i2 at stage m). */
        for (int o1 = 0; o1 < N; ++o1)
            for (int v2 = 0; v2 < V; ++v2)
                for (int sg2 = 0; sg2 < S; ++sg2) {
                    const int a2 = sg2 + (v2 << (m + 1)), b2 = a2 + S;
                    const int q0 = (sg2 << 1) + (v2 << (m + 1)), q1 = q0 + 1;
                    bad |= drto_undo_half(fb + ((size_t)o1 * N + a2) * W,
                                          fb + ((size_t)o1 * N + b2) * W,
                                          fa + ((size_t)o1 * N + q0) * W,
                                          fa + ((size_t)o1 * N + q1) * W, W, sg2, scratch);
                }
        /* Undo the s1 half-stage: fb rows (o1, i2) -> fa rows (i1, i2). */
        for (int i2 = 0; i2 < N; ++i2)
            for (int v1 = 0; v1 < V; ++v1)
                for (int sg1 = 0; sg1 < S; ++sg1) {
                    const int a1 = sg1 + (v1 << (m + 1)), b1 = a1 + S;
                    const int q0 = (sg1 << 1) + (v1 << (m + 1)), q1 = q0 + 1;
                    bad |= drto_undo_half(fa + ((size_t)a1 * N + i2) * W,
                                          fa + ((size_t)b1 * N + i2) * W,
                                          fb + ((size_t)q0 * N + i2) * W,
                                          fb + ((size_t)q1 * N + i2) * W, W, sg1, scratch);
                }
    }
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y) {
            const uint32_t* row = fa + ((size_t)x * N + y) * W;
            for (int d = 0; d < W; ++d) {
                if (d < 2 * N) { if (row[d] != 0) bad = 1; }
                else g[((size_t)x * N + y) * N + (d - 2 * N)] = row[d];
            }
        }
    free(fa); free(fb); free(scratch);
    return bad ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Lines, definition eq.(3DfDJT): brute-force scatter.                       */
/*   J[s1][s2][d1][d2] = sum_x g(x, l_{s1}(x) + d1 - N, l_{s2}(x) + d2 - N)   */
/* ------------------------------------------------------------------------ */
void drto_lines_brute_i64(int N, const int64_t* g, int64_t* J) {
    const int n = ilog2(N), D = 2 * N;
    memset(J, 0, sizeof(int64_t) * (size_t)N * N * D * D);
    for (int s1 = 0; s1 < N; ++s1)
        for (int s2 = 0; s2 < N; ++s2)
            for (int x = 0; x < N; ++x) {
                const int64_t l1 = drto_lline(n, s1, x), l2 = drto_lline(n, s2, x);
                for (int y = 0; y < N; ++y)
                    for (int z = 0; z < N; ++z) {
                        const int64_t d1 = y - l1 + N, d2 = z - l2 + N;
                        J[(((int64_t)s1 * N + s2) * D + d1) * D + d2] += g[((int64_t)x * N + y) * N + z];
                    }
            }
}
/* One cell of eq.(3DfDJT), gather form, int64: O(N). */
int64_t drto_lines_cell_i64(int N, const int32_t* g, int s1, int s2, int d1, int d2) {
    const int n = ilog2(N);
    int64_t acc = 0;
    for (int x = 0; x < N; ++x) {
        const int64_t y = drto_lline(n, s1, x) + d1 - N;
        const int64_t z = drto_lline(n, s2, x) + d2 - N;
        if (y >= 0 && y < N && z >= 0 && z < N) acc += g[((int64_t)x * N + y) * N + z];
    }
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Lines, Algorithm 3 (basicDJT3D) with the stage map eq.(map3DJ).           */
/* Buffers N^2 x 2N x 2N; row index holds (v: n-m bits, s1: m, s2: m, 0) as   */
/* v + (s1 << (n-m)) + (s2 << n); the volume is placed at [0:N, N:2N, N:2N]; */
/* the shifted read is 0 outside [0, 2N) on either displacement; each output */
/* is the sum of two reads.  separateS1S2 reads row s1 + (s2 << n).  The d2  */
/* loop runs innermost (memory order); iterations are independent.           */
/* ------------------------------------------------------------------------ */
int drto_lines_alg3_i32(int N, const int32_t* g_, int32_t* J_) {
    const uint32_t* g = (const uint32_t*)g_;
    uint32_t* J = (uint32_t*)J_;
    const int n = ilog2(N), D = 2 * N;
    const size_t plane = (size_t)D * D, cells = (size_t)N * N * plane;
    uint32_t* fm = (uint32_t*)calloc(cells, sizeof(uint32_t));
    uint32_t* fn = (uint32_t*)calloc(cells, sizeof(uint32_t));
    if (!fm || !fn) { free(fm); free(fn); return -1; }
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y)
            for (int z = 0; z < N; ++z)
                fm[(size_t)x * plane + (size_t)(N + y) * D + (N + z)] = g[((size_t)x * N + y) * N + z];
    for (int m = 0; m < n; ++m) {
        const int S = 1 << m, V = 1 << (n - m - 1);
        memset(fn, 0, cells * sizeof(uint32_t));
        for (int sg2 = 0; sg2 < S; ++sg2)
        for (int l2 = 0; l2 < 2; ++l2)
        for (int sg1 = 0; sg1 < S; ++sg1)
        for (int l1 = 0; l1 < 2; ++l1)
        for (int v = 0; v < V; ++v) {
            const size_t r0 = (size_t)((v << 1) + (sg1 << (n - m)) + (sg2 << n));
            const size_t r1 = r0 + 1;
            const size_t ro = (size_t)(v + (l1 << (n - m - 1)) + (sg1 << (n - m)) + (l2 << n) + (sg2 << (n + 1)));
            const int sh1 = sg1 + l1, sh2 = sg2 + l2;
            for (int d1 = 0; d1 < D; ++d1) {
                const uint32_t* p0 = fm + r0 * plane + (size_t)d1 * D;
                const int e1 = d1 + sh1;
                const uint32_t* p1 = (e1 < D) ? fm + r1 * plane + (size_t)e1 * D : NULL;
                uint32_t* po = fn + ro * plane + (size_t)d1 * D;
                for (int d2 = 0; d2 < D; ++d2) {
                    const int e2 = d2 + sh2;
                    uint32_t f1 = (p1 && e2 < D) ? p1[e2] : 0u;
                    po[d2] = p0[d2] + f1;
                }
            }
        }
        uint32_t* t = fm; fm = fn; fn = t;
    }
    for (int s1 = 0; s1 < N; ++s1)
        for (int s2 = 0; s2 < N; ++s2)
            memcpy(J + ((size_t)s1 * N + s2) * plane, fm + (size_t)(s1 + (s2 << n)) * plane,
                   plane * sizeof(uint32_t));
    free(fm); free(fn);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Lines adjoint (backprojection), definition: the transposed scatter of     */
/* eq.(3DfDJT) -- every voxel on the line of cell (s1, s2, d1, d2) receives   */
/* that cell's value:                                                        */
/*   gbar[x][y][z] = sum_{s1,s2} Jbar[s1][s2][y - l_{s1}(x) + N][z - l_{s2}(x) + N] */
/* (both displacements are always inside [1, 2N)).  int64.                   */
/* ------------------------------------------------------------------------ */
void drto_lines_adjoint_brute_i64(int N, const int64_t* Jbar, int64_t* gbar) {
    const int n = ilog2(N), D = 2 * N;
    memset(gbar, 0, sizeof(int64_t) * (size_t)N * N * N);
    for (int s1 = 0; s1 < N; ++s1)
        for (int s2 = 0; s2 < N; ++s2)
            for (int x = 0; x < N; ++x) {
                const int64_t l1 = drto_lline(n, s1, x), l2 = drto_lline(n, s2, x);
                for (int y = 0; y < N; ++y)
                    for (int z = 0; z < N; ++z) {
                        const int64_t d1 = y - l1 + N, d2 = z - l2 + N;
                        gbar[((int64_t)x * N + y) * N + z] += Jbar[(((int64_t)s1 * N + s2) * D + d1) * D + d2];
                    }
            }
}

/* ------------------------------------------------------------------------ */
/* Lines adjoint by the reversed stage loop of Algorithm 3 with              */
/* eq.(invmap3DJsummation): separateS1S2 transposed (row s1 + (s2 << n) takes */
/* Jbar[s1][s2]), then for m = n-1 .. 0 each stage-m row pair (v bit 0, v bit */
/* 1) gathers the four stage-(m+1) rows (l1, l2) it fed: bit 0 unshifted, bit */
/* 1 at (d1 - sh1, d2 - sh2) with the forward's shifts (reads below 0 are     */
/* zero); finally the volume is read back from [0:N, N:2N, N:2N].  Same row   */
/* layout as drto_lines_alg3_i32; int32 wrap.                                */
/* ------------------------------------------------------------------------ */
int drto_lines_adjoint_i32(int N, const int32_t* Jbar_, int32_t* gbar_) {
    const uint32_t* Jbar = (const uint32_t*)Jbar_;
    uint32_t* gbar = (uint32_t*)gbar_;
    const int n = ilog2(N), D = 2 * N;
    const size_t plane = (size_t)D * D, cells = (size_t)N * N * plane;
    uint32_t* fm = (uint32_t*)calloc(cells, sizeof(uint32_t));
    uint32_t* fn = (uint32_t*)calloc(cells, sizeof(uint32_t));
    if (!fm || !fn) { free(fm); free(fn); return -1; }
    for (int s1 = 0; s1 < N; ++s1)
        for (int s2 = 0; s2 < N; ++s2)
            memcpy(fm + (size_t)(s1 + (s2 << n)) * plane, Jbar + ((size_t)s1 * N + s2) * plane,
                   plane * sizeof(uint32_t));
    for (int m = n - 1; m >= 0; --m) {
        const int S = 1 << m, V = 1 << (n - m - 1);
        memset(fn, 0, cells * sizeof(uint32_t));
        for (int sg2 = 0; sg2 < S; ++sg2)
        for (int l2 = 0; l2 < 2; ++l2)
        for (int sg1 = 0; sg1 < S; ++sg1)
        for (int l1 = 0; l1 < 2; ++l1)
        for (int v = 0; v < V; ++v) {
            const size_t r0 = (size_t)((v << 1) + (sg1 << (n - m)) + (sg2 << n));
            const size_t r1 = r0 + 1;
            const size_t ro = (size_t)(v + (l1 << (n - m - 1)) + (sg1 << (n - m)) + (l2 << n) + (sg2 << (n + 1)));
            const int sh1 = sg1 + l1, sh2 = sg2 + l2;
            for (int e1 = 0; e1 < D; ++e1) {
                const uint32_t* po0 = fm + ro * plane + (size_t)e1 * D;
                const int d1 = e1 - sh1;
                const uint32_t* po1 = (d1 >= 0) ? fm + ro * plane + (size_t)d1 * D : NULL;
                uint32_t* q0 = fn + r0 * plane + (size_t)e1 * D;
                uint32_t* q1 = fn + r1 * plane + (size_t)e1 * D;
                for (int e2 = 0; e2 < D; ++e2) {
                    const int d2 = e2 - sh2;
                    q0[e2] += po0[e2];
                    if (po1 && d2 >= 0) q1[e2] += po1[d2];
                }
            }
        }
        uint32_t* t = fm; fm = fn; fn = t;
    }
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y)
            for (int z = 0; z < N; ++z)
                gbar[((size_t)x * N + y) * N + z] = fm[(size_t)x * plane + (size_t)(N + y) * D + (N + z)];
    free(fm); free(fn);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 2D DRT of lines, the basic quadrant (Section 2.1).  An image f[u][y],      */
/* N x N; output R[s][d], d in [0, 2N), the storage index with the image      */
/* embedded at d in [N, 2N), so the line is y = l_s(u) + d - N.               */
/* ------------------------------------------------------------------------ */

/* Definition (the stage-n form of eq.(our2Dfm)): brute-force scatter of     */
/* every pixel onto the one displacement it lies on for each slope.          */
/*   R[s][d] = sum_u f(u, l_s(u) + d - N)                                     */
void drto_drt2d_brute_i64(int N, const int64_t* f, int64_t* R) {
    const int n = ilog2(N), W = 2 * N;
    memset(R, 0, sizeof(int64_t) * (size_t)N * W);
    for (int s = 0; s < N; ++s)
        for (int u = 0; u < N; ++u) {
            const int64_t l = drto_lline(n, s, u);
            for (int y = 0; y < N; ++y) R[(int64_t)s * W + (y - l + N)] += f[(int64_t)u * N + y];
        }
}

/* Stage recursion eq.(map2D).  The partial transform of stage m is stored   */
/* as fm[sigma][v][d]: sigma = lambda of the m slope bits, v = lambda of the  */
/* n - m position bits still to be summed, flattened to row                   */
/* sigma * 2^(n-m) + v.  Stage 0 is the image (sigma empty, v = u), stage n   */
/* is R (v empty).  One stage prepends the slope bit s_{n-m-1} as the new     */
/* least significant bit (S = 2 sigma + s_{n-m-1}) and consumes the lowest    */
/* position bit v_m:                                                          */
/*   f^{m+1}(S | V | d) = f^m(sigma | 2V | d)                                 */
/*                      + f^m(sigma | 2V + 1 | d + s_{n-m-1} + sigma),        */
/* and s_{n-m-1} + sigma = floor((S + 1) / 2).  Reads past 2N are zero.       */
#define DRTO_MAP2D_BODY(T)                                                          \
    const int n = ilog2(N), W = 2 * N;                                              \
    const size_t cells = (size_t)N * W;                                             \
    T* fm = (T*)calloc(cells, sizeof(T));                                           \
    T* fn = (T*)calloc(cells, sizeof(T));                                           \
    if (!fm || !fn) { free(fm); free(fn); return -1; }                              \
    for (int u = 0; u < N; ++u)                                                     \
        for (int y = 0; y < N; ++y) fm[(size_t)u * W + N + y] = (T)f[(size_t)u * N + y]; \
    for (int m = 0; m < n; ++m) {                                                   \
        const int Vn = 1 << (n - m - 1);  /* position values after the stage */    \
        for (int S = 0; S < (2 << m); ++S)                                          \
            for (int V = 0; V < Vn; ++V) {                                          \
                const int sigma = S >> 1, sh = (S + 1) >> 1;                        \
                const T* lo = fm + ((size_t)sigma * (2 * Vn) + 2 * V) * W;          \
                const T* hi = fm + ((size_t)sigma * (2 * Vn) + 2 * V + 1) * W;      \
                T* out = fn + ((size_t)S * Vn + V) * W;                             \
                for (int d = 0; d < W; ++d)                                         \
                    out[d] = lo[d] + ((d + sh < W) ? hi[d + sh] : (T)0);            \
            }                                                                       \
        T* t = fm; fm = fn; fn = t;                                                 \
    }                                                                               \
    memcpy(R, fm, cells * sizeof(T));                                               \
    free(fm); free(fn);                                                             \
    return 0;

int drto_drt2d_map2d_i32(int N, const int32_t* f, int32_t* R_) {
    uint32_t* R = (uint32_t*)R_;
    DRTO_MAP2D_BODY(uint32_t)
}
int drto_drt2d_map2d_f64(int N, const double* f, double* R) {
    DRTO_MAP2D_BODY(double)
}
