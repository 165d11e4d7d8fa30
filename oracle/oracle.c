/*
 * Plain FP64 CPU oracle for the solid-angle labeling method.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code with the CUDA path.
 *
 * What it computes (Sec. 2.1.3, Eq. 1): for a query point p and a closed
 * triangulated surface dS, the solid angle that dS subtends at p,
 *
 *     Omega(p) = integral over dS of (r - p) . n / |r - p|^3 dA,
 *
 * so that s = Omega / (4 pi) is the ratio the paper calls s_i.  (The printed
 * integrand lacks the 1/|r - p|^3 factor; without it the integral is not a
 * solid angle, so the text's definition of s_i as a solid-angle ratio is
 * followed.)  The integral over one flat triangle has the closed form of Van
 * Oosterom and Strackee (IEEE Trans. Biomed. Eng. 30(2), 1983):
 *
 *     tan(Omega_t / 2) = N / D,
 *     N = R1 . (R2 x R3),
 *     D = r1 r2 r3 + (R1 . R2) r3 + (R1 . R3) r2 + (R2 . R3) r1,
 *
 * with R_k = v_k - p the vectors from p to the triangle's vertices (in the
 * triangle's own vertex order) and r_k = |R_k|.  Omega_t = 2 atan2(N, D) and
 * Omega(p) is the sum over the triangles, taken in index order, in double.
 *
 * Parity pins: closed forms (octant, cube centre, regular-tetrahedron
 * centroid, unit sphere), L'Huilier's spherical-excess theorem on random
 * triangles, the integer winding invariant and ray-parity crossing counts;
 * see tests/test_oracle_pins.py.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fast-math, so
 * libm atan2 and sqrt are used as written).
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Solid angle of one triangle (a, b, c) seen from p (Van Oosterom-Strackee). */
static double triangle_solid_angle(const double *p, const double *a,
                                   const double *b, const double *c)
{
    double R1[3], R2[3], R3[3];
    for (int k = 0; k < 3; ++k) {
        R1[k] = a[k] - p[k];
        R2[k] = b[k] - p[k];
        R3[k] = c[k] - p[k];
    }
    double r1 = sqrt(R1[0] * R1[0] + R1[1] * R1[1] + R1[2] * R1[2]);
    double r2 = sqrt(R2[0] * R2[0] + R2[1] * R2[1] + R2[2] * R2[2]);
    double r3 = sqrt(R3[0] * R3[0] + R3[1] * R3[1] + R3[2] * R3[2]);
    /* R2 x R3 */
    double cx = R2[1] * R3[2] - R2[2] * R3[1];
    double cy = R2[2] * R3[0] - R2[0] * R3[2];
    double cz = R2[0] * R3[1] - R2[1] * R3[0];
    double N = R1[0] * cx + R1[1] * cy + R1[2] * cz;
    double d12 = R1[0] * R2[0] + R1[1] * R2[1] + R1[2] * R2[2];
    double d13 = R1[0] * R3[0] + R1[1] * R3[1] + R1[2] * R3[2];
    double d23 = R2[0] * R3[0] + R2[1] * R3[1] + R2[2] * R3[2];
    double D = r1 * r2 * r3 + d12 * r3 + d13 * r2 + d23 * r1;
    return 2.0 * atan2(N, D);
}

/*
 * omega[i] = sum over triangles t (index order) of Omega_t(points[i]).
 *   points: n x 3 doubles; verts: nv x 3 doubles; tris: nt x 3 int32 (0-based)
 *   nthreads <= 0 uses the OpenMP default.
 * Returns 0, or -1 when a triangle index is out of range (nothing written).
 */
int oracle_omega(const double *points, int64_t n, const double *verts, int64_t nv,
                 const int32_t *tris, int64_t nt, double *omega, int nthreads)
{
    for (int64_t t = 0; t < 3 * nt; ++t)
        if (tris[t] < 0 || tris[t] >= nv)
            return -1;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        const double *p = points + 3 * i;
        double s = 0.0;
        for (int64_t t = 0; t < nt; ++t) {
            const int32_t *f = tris + 3 * t;
            s += triangle_solid_angle(p, verts + 3 * (int64_t)f[0], verts + 3 * (int64_t)f[1],
                                      verts + 3 * (int64_t)f[2]);
        }
        omega[i] = s;
    }
    return 0;
}

/* Per-triangle solid angles for one point (used by the closed-form pins). */
int oracle_triangle_terms(const double *p, const double *verts, int64_t nv,
                          const int32_t *tris, int64_t nt, double *terms)
{
    for (int64_t t = 0; t < 3 * nt; ++t)
        if (tris[t] < 0 || tris[t] >= nv)
            return -1;
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t *f = tris + 3 * t;
        terms[t] = triangle_solid_angle(p, verts + 3 * (int64_t)f[0], verts + 3 * (int64_t)f[1],
                                        verts + 3 * (int64_t)f[2]);
    }
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
