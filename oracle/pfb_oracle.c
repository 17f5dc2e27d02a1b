/*
 * FP64 oracle for the wide-field measurement operator (test infrastructure
 * only: the product path never links or calls this file).
 *
 * Plain direct evaluation of the measurement equation of Section 2 (Eq. 1):
 * the visibility of channel nu on row d is
 *
 *     V[d,nu] = sum_{i,j} x[b(nu),i,j] / n_ij * exp(-2 pi i (u l_i + v m_j + w (n_ij - 1)))
 *
 * with (u,v,w) = uvw_d * f_nu / c (wavelengths), l_i = l0 + (i - nx/2) dl,
 * m_j = m0 + (j - ny/2) dm, n_ij = sqrt(1 - l_i^2 - m_j^2), and b(nu) the imaging
 * band of channel nu (Section 2: n_b bands, n_b << n_nu).  The adjoint
 * R^dagger used in Eq. 3 is the transpose under the real inner products
 * <a,b> = Re sum conj(a) b on visibilities and <x,z> = sum x z on images:
 *
 *     (R^dagger y)[b,i,j] = Re sum_{nu in b} sum_d y[d,nu] exp(+2 pi i phi) / n_ij.
 *
 * Every phase is reduced in FP64 (phi - rint(phi), in cycles) before sin/cos.
 * No gridding, no FFT, no approximation: the cost is O(visibilities x pixels).
 *
 * Flags: bit 0 drops the 1/n factor, bit 1 drops the w (n-1) term.  Both are
 * test switches that turn the operator into a plain 2-D non-uniform DFT.
 *
 * (l0, m0) places the image centre away from the phase centre: the image is then
 * one facet of a larger field, and the operator is still the definition above with
 * the facet's absolute l, m (the phase centre of the data does not move).  With
 * l0 = m0 = 0 the image is centred on the phase centre.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_NO_DIVIDE_BY_N 1u
#define ORACLE_NO_WTERM 2u

static const double C_LIGHT = 299792458.0;
static const double TWO_PI = 6.283185307179586476925286766559;

/* exp(sign * 2 pi i phi) with phi in cycles, reduced to [-1/2, 1/2] first */
static inline void cis_cycles(double phi, double sign, double *re, double *im) {
    double r = phi - rint(phi);
    double a = TWO_PI * r;
    *re = cos(a);
    *im = sign * sin(a);
}

static inline void pixel_lmn(int i, int j, int nx, int ny, double dl, double dm, double l0, double m0,
                             unsigned flags, double *l, double *m, double *nm1, double *ninv) {
    *l = l0 + (double)(i - nx / 2) * dl;
    *m = m0 + (double)(j - ny / 2) * dm;
    double s = 1.0 - (*l) * (*l) - (*m) * (*m);
    double n = sqrt(s);
    /* n - 1 written as -(l^2+m^2)/(1+n): no cancellation near the phase centre */
    *nm1 = (flags & ORACLE_NO_WTERM) ? 0.0 : -((*l) * (*l) + (*m) * (*m)) / (1.0 + n);
    *ninv = (flags & ORACLE_NO_DIVIDE_BY_N) ? 1.0 : 1.0 / n;
}

/*
 * R (Eq. 1): image [nband][nx][ny] -> vis [nrow][nchan] complex (re,im pairs).
 * If rows != NULL only the nsel listed rows are evaluated and vis is [nsel][nchan].
 */
void oracle_degrid(int nx, int ny, double dl, double dm, double l0, double m0, int nband, int64_t nrow, int nchan,
                   const double *uvw, const double *freq, const int32_t *band_of_chan,
                   const double *image, unsigned flags, int64_t nsel, const int64_t *rows,
                   double *vis) {
    const int64_t npix = (int64_t)nx * ny;
    /* list the non-zero pixels of each band once: the sky models are sparse */
    int64_t *cnt = (int64_t *)calloc((size_t)nband, sizeof(int64_t));
    for (int b = 0; b < nband; ++b)
        for (int64_t p = 0; p < npix; ++p)
            if (image[b * npix + p] != 0.0) cnt[b]++;
    double **tab = (double **)calloc((size_t)nband, sizeof(double *));
    for (int b = 0; b < nband; ++b) {
        tab[b] = (double *)malloc((size_t)(cnt[b] > 0 ? cnt[b] : 1) * 4 * sizeof(double));
        int64_t k = 0;
        for (int64_t p = 0; p < npix; ++p) {
            double xv = image[b * npix + p];
            if (xv == 0.0) continue;
            int i = (int)(p / ny), j = (int)(p % ny);
            double l, m, nm1, ninv;
            pixel_lmn(i, j, nx, ny, dl, dm, l0, m0, flags, &l, &m, &nm1, &ninv);
            tab[b][4 * k + 0] = l;
            tab[b][4 * k + 1] = m;
            tab[b][4 * k + 2] = nm1;
            tab[b][4 * k + 3] = xv * ninv;
            ++k;
        }
    }
    const int64_t nout = rows ? nsel : nrow;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nout; ++r) {
        const int64_t d = rows ? rows[r] : r;
        for (int c = 0; c < nchan; ++c) {
            const double s = freq[c] / C_LIGHT;
            const double u = uvw[3 * d + 0] * s, v = uvw[3 * d + 1] * s, w = uvw[3 * d + 2] * s;
            const int b = band_of_chan[c];
            const double *t = tab[b];
            double are = 0.0, aim = 0.0;
            for (int64_t k = 0; k < cnt[b]; ++k) {
                double phi = u * t[4 * k] + v * t[4 * k + 1] + w * t[4 * k + 2];
                double cr, ci;
                cis_cycles(phi, -1.0, &cr, &ci);
                are += t[4 * k + 3] * cr;
                aim += t[4 * k + 3] * ci;
            }
            vis[2 * (r * nchan + c) + 0] = are;
            vis[2 * (r * nchan + c) + 1] = aim;
        }
    }
    for (int b = 0; b < nband; ++b) free(tab[b]);
    free(tab);
    free(cnt);
}

/*
 * R^dagger Sigma^-1 (Eq. 3): vis [nrow][nchan] complex, wgt [nrow][nchan] (NULL = ones)
 * -> image.  If pix != NULL only the npix listed flat indices b*nx*ny + i*ny + j are
 * evaluated and out is [npix]; otherwise out is the full [nband][nx][ny] cube.
 */
void oracle_grid(int nx, int ny, double dl, double dm, double l0, double m0, int nband, int64_t nrow, int nchan,
                 const double *uvw, const double *freq, const int32_t *band_of_chan,
                 const double *vis, const double *wgt, unsigned flags, int64_t npix,
                 const int64_t *pix, double *out) {
    const int64_t ncube = (int64_t)nband * nx * ny;
    const int64_t nout = pix ? npix : ncube;
    /* per-channel scaled frequencies, reused by every pixel */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nout; ++q) {
        const int64_t p = pix ? pix[q] : q;
        const int b = (int)(p / ((int64_t)nx * ny));
        const int64_t pp = p % ((int64_t)nx * ny);
        const int i = (int)(pp / ny), j = (int)(pp % ny);
        double l, m, nm1, ninv;
        pixel_lmn(i, j, nx, ny, dl, dm, l0, m0, flags, &l, &m, &nm1, &ninv);
        double acc = 0.0;
        for (int c = 0; c < nchan; ++c) {
            if (band_of_chan[c] != b) continue;
            const double s = freq[c] / C_LIGHT;
            for (int64_t d = 0; d < nrow; ++d) {
                const double u = uvw[3 * d + 0] * s, v = uvw[3 * d + 1] * s, w = uvw[3 * d + 2] * s;
                double phi = u * l + v * m + w * nm1;
                double cr, ci;
                cis_cycles(phi, +1.0, &cr, &ci);
                const int64_t k = d * nchan + c;
                const double wt = wgt ? wgt[k] : 1.0;
                /* Re[(yr + i yi)(cr + i ci)] = yr cr - yi ci */
                acc += wt * (vis[2 * k] * cr - vis[2 * k + 1] * ci);
            }
        }
        out[q] = acc * ninv;
    }
}

/*
 * Sum of the weights of each band (the PSF peak; used to normalise the step).
 */
void oracle_wsum(int nband, int64_t nrow, int nchan, const int32_t *band_of_chan,
                 const double *wgt, double *wsum) {
    for (int b = 0; b < nband; ++b) wsum[b] = 0.0;
    for (int64_t d = 0; d < nrow; ++d)
        for (int c = 0; c < nchan; ++c)
            wsum[band_of_chan[c]] += wgt ? wgt[d * nchan + c] : 1.0;
}

/*
 * Linear convolution with the PSF by direct summation (Eq. 4's I^psf * x):
 *   y[b,i,j] = sum_{i',j'} psf[b, i-i'+nx, j-j'+ny] x[b,i',j'],
 * psf is [nband][2nx][2ny] with its centre at (nx, ny).  O(n_p^2): tiny images only.
 */
void oracle_psf_conv_direct(int nx, int ny, int nband, const double *psf, const double *x,
                            double *y) {
    const int64_t NX = 2 * (int64_t)nx, NY = 2 * (int64_t)ny;
#pragma omp parallel for collapse(2) schedule(static)
    for (int b = 0; b < nband; ++b)
        for (int i = 0; i < nx; ++i) {
            for (int j = 0; j < ny; ++j) {
                double acc = 0.0;
                for (int ip = 0; ip < nx; ++ip)
                    for (int jp = 0; jp < ny; ++jp)
                        acc += psf[(int64_t)b * NX * NY + (int64_t)(i - ip + nx) * NY + (j - jp + ny)] *
                               x[((int64_t)b * nx + ip) * ny + jp];
                y[((int64_t)b * nx + i) * ny + j] = acc;
            }
        }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
