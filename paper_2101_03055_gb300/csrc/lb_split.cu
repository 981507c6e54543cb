// A lattice split into slabs of whole rows, all on one device (cdf_split_*).
//
// The update of a node reads only its nearest neighbours' post-collision
// populations of the previous step (Eqs. evolution12 and evolution3 with
// streaming, Sec. 2), so a slab advances exactly like its rows of the whole
// lattice when its halo rows hold, before every step, the populations that
// cross the cut from the neighbouring slab.  This driver is written against the
// public per-slab calls only -- cdf_lb_step, cdf_lb_halo_pack/unpack,
// cdf_lb_mass, cdf_lb_snapshot, cdf_lb_change_sums -- which are the calls a
// one-slab-per-GPU process makes, with the packed rows moved by its collective
// library instead of a device copy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/cdf_lb.h"
#include "lb_internal.h"

using cdflb::report_error;

struct cdf_split {
    int nx = 0, ny = 0, m = 0, n = 0;
    bool periodic_y = false;
    std::vector<cdf_lb *> slab;
    std::vector<int> y0, rows, halo, origin, lny;
    float *bufs = nullptr;  // per cut: [up][3 + m][nx] and [down][3 + m][nx]
    int ncuts = 0;
    cudaStream_t user = nullptr;
};

namespace {

void split_release(cdf_split *s) {
    if (!s) return;
    for (cdf_lb *h : s->slab) cdf_lb_destroy(h);
    if (s->bufs) cudaFree(s->bufs);
    delete s;
}

// Lower and upper slab of cut c (cut c lies above slab c; the last cut of a
// periodic axis joins the top slab to slab 0).
void cut_slabs(const cdf_split *s, int c, int *lo, int *hi) {
    *lo = c;
    *hi = (c + 1) % s->n;
}

// Moves the crossing rows of every cut: the lower slab's last updated row goes
// up into the upper slab's south halo row, the upper slab's first updated row
// down into the lower slab's north halo row.
cdf_status exchange(cdf_split *s) {
    const size_t row = (size_t)(3 + s->m) * s->nx;
    for (int c = 0; c < s->ncuts; ++c) {
        int lo, hi;
        cut_slabs(s, c, &lo, &hi);
        float *up = s->bufs + 2 * c * row, *down = up + row;
        cdf_status st;
        if ((st = cdf_lb_halo_pack(s->slab[lo], 1, up)) != CDF_OK) return st;
        if ((st = cdf_lb_halo_pack(s->slab[hi], 0, down)) != CDF_OK) return st;
        if ((st = cdf_lb_halo_unpack(s->slab[hi], 0, up)) != CDF_OK) return st;
        if ((st = cdf_lb_halo_unpack(s->slab[lo], 1, down)) != CDF_OK) return st;
    }
    return CDF_OK;
}

}  // namespace

extern "C" {

cdf_status cdf_split_create(const cdf_grid *grid, int m, const cdf_diffusion *dif, double nu,
                            const cdf_source *src, const cdf_force *frc, const cdf_boundaries *bc,
                            const cdf_options *opt, int nslabs, cdf_split **out) {
    if (!out) return report_error(CDF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid || !bc || !opt) return report_error(CDF_EINVAL, "NULL argument");
    if (opt->halo_rows || opt->origin_y || opt->ny_global)
        return report_error(CDF_EINVAL, "halo_rows, origin_y and ny_global are set by the split: pass 0");
    if (m < 1 || m > CDF_MAX_M) return report_error(CDF_EINVAL, "m must be in [1, 4]");
    const bool periodic = bc->south.kind == CDF_BC_PERIODIC;
    if (nslabs < 2 || nslabs > grid->ny || (periodic && grid->ny < 2 * nslabs))
        return report_error(CDF_EINVAL, "nslabs must be in [2, ny] (ny >= 2 nslabs on a periodic y axis)");
    cdf_split *s = new (std::nothrow) cdf_split;
    if (!s) return report_error(CDF_ENOMEM, "host allocation failed");
    s->nx = grid->nx;
    s->ny = grid->ny;
    s->m = m;
    s->n = nslabs;
    s->periodic_y = periodic;
    s->user = static_cast<cudaStream_t>(opt->cuda_stream);
    s->ncuts = periodic ? nslabs : nslabs - 1;
    int y = 0;
    for (int k = 0; k < nslabs; ++k) {
        const int r = grid->ny / nslabs + (k < grid->ny % nslabs ? 1 : 0);
        const int hl = periodic ? 3 : ((k > 0 ? 1 : 0) | (k < nslabs - 1 ? 2 : 0));
        s->y0.push_back(y);
        s->rows.push_back(r);
        s->halo.push_back(hl);
        s->origin.push_back(y - (hl & 1));
        s->lny.push_back(r + (hl & 1) + (hl >> 1));
        y += r;
    }
    for (int k = 0; k < nslabs; ++k) {
        cdf_options o = *opt;
        o.halo_rows = s->halo[k];
        o.origin_y = s->origin[k];
        o.ny_global = grid->ny;
        if (o.temporal == 0) o.temporal = -1;  // one step per launch
        if (o.resident == 0) o.resident = -1;
        const cdf_grid g{grid->nx, s->lny[k]};
        cdf_lb *h = nullptr;
        cdf_status st = cdf_lb_create(&g, m, dif, nu, src, frc, bc, &o, &h);
        if (st != CDF_OK) {
            split_release(s);
            return st;
        }
        s->slab.push_back(h);
    }
    const size_t bytes = (size_t)2 * s->ncuts * (3 + m) * grid->nx * sizeof(float);
    if (cudaMalloc((void **)&s->bufs, bytes) != cudaSuccess) {
        cudaGetLastError();
        split_release(s);
        return report_error(CDF_ENOMEM, "device allocation of the halo buffers failed");
    }
    *out = s;
    return CDF_OK;
}

cdf_status cdf_split_init_moments(cdf_split *s, const double *phi, const double *u, const double *p) {
    if (!s || !phi || !u) return report_error(CDF_EINVAL, "NULL argument");
    const size_t N = (size_t)s->nx * s->ny;
    for (int k = 0; k < s->n; ++k) {
        // the slab's rows of the whole lattice, halo rows included (wrapped on a
        // periodic axis), so the halo rows start from their neighbours' state
        const size_t n = (size_t)s->nx * s->lny[k];
        std::vector<double> lphi((size_t)s->m * n), lu(2 * n), lp(p ? n : 0);
        for (int ly = 0; ly < s->lny[k]; ++ly) {
            const int gy = ((s->origin[k] + ly) % s->ny + s->ny) % s->ny;
            const size_t src = (size_t)gy * s->nx, dst = (size_t)ly * s->nx;
            for (int a = 0; a < s->m; ++a) std::memcpy(&lphi[a * n + dst], &phi[a * N + src], s->nx * 8);
            for (int c = 0; c < 2; ++c) std::memcpy(&lu[c * n + dst], &u[c * N + src], s->nx * 8);
            if (p) std::memcpy(&lp[dst], &p[src], s->nx * 8);
        }
        cdf_status st = cdf_lb_init_moments(s->slab[k], lphi.data(), lu.data(), p ? lp.data() : nullptr);
        if (st != CDF_OK) return st;
    }
    return exchange(s);
}

cdf_status cdf_split_step(cdf_split *s, long long n) {
    if (!s) return report_error(CDF_EINVAL, "NULL handle");
    if (n < 0) return report_error(CDF_EINVAL, "n must be >= 0");
    for (long long i = 0; i < n; ++i) {
        for (cdf_lb *h : s->slab) {
            cdf_status st = cdf_lb_step(h, 1);
            if (st != CDF_OK) return st;
        }
        cdf_status st = exchange(s);
        if (st != CDF_OK) return st;
    }
    return CDF_OK;
}

cdf_status cdf_split_moments(cdf_split *s, double *host_out) {
    if (!s || !host_out) return report_error(CDF_EINVAL, "NULL argument");
    const size_t N = (size_t)s->nx * s->ny;
    for (int k = 0; k < s->n; ++k) {
        const size_t n = (size_t)s->nx * s->lny[k];
        std::vector<double> loc((size_t)(s->m + 3) * n);
        cdf_status st = cdf_lb_moments(s->slab[k], loc.data());
        if (st != CDF_OK) return st;
        const int first = s->halo[k] & 1;
        for (int f = 0; f < s->m + 3; ++f)
            std::memcpy(&host_out[f * N + (size_t)s->y0[k] * s->nx], &loc[f * n + (size_t)first * s->nx],
                        (size_t)s->rows[k] * s->nx * 8);
    }
    return CDF_OK;
}

cdf_status cdf_split_mass(cdf_split *s, double *sums) {
    if (!s || !sums) return report_error(CDF_EINVAL, "NULL argument");
    for (int a = 0; a < s->m; ++a) sums[a] = 0.0;
    for (cdf_lb *h : s->slab) {
        double q[CDF_MAX_M];
        cdf_status st = cdf_lb_mass(h, q);
        if (st != CDF_OK) return st;
        for (int a = 0; a < s->m; ++a) sums[a] += q[a];
    }
    return CDF_OK;
}

cdf_status cdf_split_run_to_steady(cdf_split *s, double tol, long long check_every, long long max_steps,
                                   long long *steps_taken, double *residual) {
    if (!s) return report_error(CDF_EINVAL, "NULL handle");
    if (check_every < 1 || max_steps < 0 || !(tol > 0.0))
        return report_error(CDF_EINVAL, "bad tol / check_every / max_steps");
    const int m = s->m, nq = 3 * m + 5;
    long long taken = 0;
    double R = INFINITY;
    cdf_status result = CDF_ENOTCONVERGED;
    while (taken < max_steps) {
        cdf_status st;
        for (cdf_lb *h : s->slab)
            if ((st = cdf_lb_snapshot(h)) != CDF_OK) return st;
        const long long k = std::min(check_every, max_steps - taken);
        if ((st = cdf_split_step(s, k)) != CDF_OK) return st;
        taken += k;
        // the slabs' FP64 sums added together: the whole lattice's sums (the
        // all-reduce of a one-slab-per-GPU run)
        double q[3 * CDF_MAX_M + 5] = {0};
        for (cdf_lb *h : s->slab) {
            double qs[3 * CDF_MAX_M + 5];
            if ((st = cdf_lb_change_sums(h, qs)) != CDF_OK) return st;
            for (int j = 0; j < nq; ++j) q[j] += qs[j];
        }
        if (q[3 * m + 4] > 0) { result = CDF_EUNSTABLE; break; }
        R = 0.0;
        for (int f = 0; f < m + 2; ++f) R = std::max(R, q[m + f] / std::max(q[2 * m + 2 + f], 1e-300));
        if (k == check_every && R < tol) { result = CDF_OK; break; }
    }
    if (steps_taken) *steps_taken = taken;
    if (residual) *residual = R;
    if (result == CDF_EUNSTABLE) return report_error(CDF_EUNSTABLE, "non-finite moments in a slab");
    if (result == CDF_ENOTCONVERGED) return report_error(CDF_ENOTCONVERGED, "residual above tol after max_steps");
    return CDF_OK;
}

cdf_status cdf_split_slab(const cdf_split *s, int k, cdf_lb **slab, int *y0, int *rows) {
    if (!s || k < 0 || k >= s->n) return report_error(CDF_EINVAL, "no such slab");
    if (slab) *slab = s->slab[k];
    if (y0) *y0 = s->y0[k];
    if (rows) *rows = s->rows[k];
    return CDF_OK;
}

void cdf_split_destroy(cdf_split *s) { split_release(s); }

}  // extern "C"
