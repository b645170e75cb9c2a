/*
 * Truth trajectories of the synthetic-input generator in an axisymmetric
 * (r, z) field map: the generator's own classical Runge-Kutta (RK4) on the
 * 6-D state (position, unit direction) with a fixed step ds, the field
 * interpolated bilinearly in (r, z) of the FP32 samples.  This is input
 * synthesis only (the truth the synthetic hits come from), written out here
 * because the same loop in Python dominates event generation; it holds none
 * of the track finder's arithmetic.  Build with -ffp-contract=off so that
 * every machine rounds the same operations in the same order.
 */
#include <math.h>

typedef struct {
    const float* bz; /* [nr][nz] */
    const float* br;
    int nr, nz;
    double r_min, z_min, dr, dz;
} synth_map;

static void field_at(const synth_map* f, double x, double y, double z, double* bx, double* by, double* bz) {
    double rho = sqrt(x * x + y * y);
    double rc = rho < f->r_min ? f->r_min : rho;
    double rmax = f->r_min + f->dr * (f->nr - 1), zmax = f->z_min + f->dz * (f->nz - 1);
    if (rc > rmax) rc = rmax;
    double zc = z < f->z_min ? f->z_min : z;
    if (zc > zmax) zc = zmax;
    double u = (rc - f->r_min) / f->dr, v = (zc - f->z_min) / f->dz;
    int i = (int)u, j = (int)v;
    if (i > f->nr - 2) i = f->nr - 2;
    if (j > f->nz - 2) j = f->nz - 2;
    u -= i;
    v -= j;
    double w00 = (1 - u) * (1 - v), w10 = u * (1 - v), w01 = (1 - u) * v, w11 = u * v;
    const long a = (long)i * f->nz + j, b = (long)(i + 1) * f->nz + j;
    double z_ = w00 * (double)f->bz[a] + w10 * (double)f->bz[b] + w01 * (double)f->bz[a + 1] + w11 * (double)f->bz[b + 1];
    double r_ = w00 * (double)f->br[a] + w10 * (double)f->br[b] + w01 * (double)f->br[a + 1] + w11 * (double)f->br[b + 1];
    *bz = z_;
    if (rho < 1e-12) {
        *bx = 0.0;
        *by = 0.0;
    } else {
        *bx = r_ * x / rho;
        *by = r_ * y / rho;
    }
}

static void accel(const synth_map* f, double lam, double x, double y, double z, double tx, double ty, double tz,
                  double a[3]) {
    double bx, by, bz;
    field_at(f, x, y, z, &bx, &by, &bz);
    a[0] = lam * (ty * bz - tz * by);
    a[1] = lam * (tz * bx - tx * bz);
    a[2] = lam * (tx * by - ty * bx);
}

/* Samples pos/dirs [n][3] from r0, t0 every ds mm until |z| > z_stop or
 * rho > r_stop (that sample included) or n samples; returns the count. */
int synth_track_map(const float* bz, const float* br, int nr, int nz, double r_min, double z_min, double dr,
                    double dz, double lam, const double* r0, const double* t0, double ds, int n, double z_stop,
                    double r_stop, double* pos, double* dirs) {
    synth_map f = {bz, br, nr, nz, r_min, z_min, dr, dz};
    double x = r0[0], y = r0[1], z = r0[2], tx = t0[0], ty = t0[1], tz = t0[2];
    double h2 = 0.5 * ds;
    for (int i = 0; i < n; ++i) {
        pos[3 * i] = x;
        pos[3 * i + 1] = y;
        pos[3 * i + 2] = z;
        dirs[3 * i] = tx;
        dirs[3 * i + 1] = ty;
        dirs[3 * i + 2] = tz;
        double a1[3], a2[3], a3[3], a4[3], b2[3], b3[3], b4[3];
        accel(&f, lam, x, y, z, tx, ty, tz, a1);
        accel(&f, lam, x + h2 * tx, y + h2 * ty, z + h2 * tz, tx + h2 * a1[0], ty + h2 * a1[1], tz + h2 * a1[2], a2);
        b2[0] = tx + h2 * a1[0];
        b2[1] = ty + h2 * a1[1];
        b2[2] = tz + h2 * a1[2];
        accel(&f, lam, x + h2 * b2[0], y + h2 * b2[1], z + h2 * b2[2], tx + h2 * a2[0], ty + h2 * a2[1],
              tz + h2 * a2[2], a3);
        b3[0] = tx + h2 * a2[0];
        b3[1] = ty + h2 * a2[1];
        b3[2] = tz + h2 * a2[2];
        b4[0] = tx + ds * a3[0];
        b4[1] = ty + ds * a3[1];
        b4[2] = tz + ds * a3[2];
        accel(&f, lam, x + ds * b3[0], y + ds * b3[1], z + ds * b3[2], b4[0], b4[1], b4[2], a4);
        double c = ds / 6;
        x += c * (tx + 2 * b2[0] + 2 * b3[0] + b4[0]);
        y += c * (ty + 2 * b2[1] + 2 * b3[1] + b4[1]);
        z += c * (tz + 2 * b2[2] + 2 * b3[2] + b4[2]);
        tx += c * (a1[0] + 2 * a2[0] + 2 * a3[0] + a4[0]);
        ty += c * (a1[1] + 2 * a2[1] + 2 * a3[1] + a4[1]);
        tz += c * (a1[2] + 2 * a2[2] + 2 * a3[2] + a4[2]);
        if (fabs(z) > z_stop || sqrt(x * x + y * y) > r_stop) {
            if (i + 1 < n) {
                pos[3 * (i + 1)] = x;
                pos[3 * (i + 1) + 1] = y;
                pos[3 * (i + 1) + 2] = z;
                dirs[3 * (i + 1)] = tx;
                dirs[3 * (i + 1) + 1] = ty;
                dirs[3 * (i + 1) + 2] = tz;
                return i + 2;
            }
            return n;
        }
    }
    return n;
}
