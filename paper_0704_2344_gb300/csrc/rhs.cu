// Right-hand side of Eq. 4 for incident plane waves:
//   b(W) = G(W, H_i) - int_Sext W . (n x curl H_i) ds,
// with G the weak Engquist-Majda form of Eq. 3 (the same integrated-by-parts
// form as the left-hand side) and H_i = p_hat H0 exp(-j k0 k_hat . r),
// curl H_i = -j k0 k_hat x H_i.  One thread per (active node, wave) gathers
// the outer faces around its node (2x2 Gauss points per face), so the sum is
// deterministic and atomic-free.
#include "fe_internal.cuh"

namespace fe {

struct Wave {
    double k[3], p[3];
    double ar, ai;
};

__global__ void k_rhs(int nx, int ny, int nz, double hx, double hy, double hz, double ox, double oy, double oz,
                      double k0, double sigma, const int* __restrict__ node_id, int n_act,
                      const Wave* __restrict__ waves, int nrhs, unsigned abc, unsigned planes,
                      const uint8_t* __restrict__ mat, int form_e, double2* __restrict__ B) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_act * nrhs) return;
    const int r = (int)(t / nrhs), w = (int)(t - (int64_t)r * nrhs);
    const int id = node_id[r];
    const int c[3] = {id % (nx + 1), (id / (nx + 1)) % (ny + 1), id / ((nx + 1) * (ny + 1))};
    const int dim[3] = {nx, ny, nz};
    const double h[3] = {hx, hy, hz};
    const double org[3] = {ox, oy, oz};
    const Wave wv = waves[w];
    double br[3] = {0, 0, 0}, bi[3] = {0, 0, 0};
    const double g0 = 0.5 - 0.5 / sqrt(3.0), g1 = 0.5 + 0.5 / sqrt(3.0);
    for (int f = 0; f < 6; ++f) {
        const int nu = f >> 1, side = f & 1;
        if (c[nu] != (side ? dim[nu] : 0) || !((abc >> f) & 1u)) continue;  // absorbing faces only
        const int t1 = nu == 0 ? 1 : 0, t2 = nu == 2 ? 1 : 2;
        const double nsgn = side ? 1.0 : -1.0;
        // n . k_hat and the element coordinate along the normal
        const double nk = nsgn * wv.k[nu];
        const int e_nu = side ? dim[nu] - 1 : 0;
        for (int s2 = 0; s2 < 2; ++s2) {
            const int e2 = c[t2] - 1 + s2;
            if (e2 < 0 || e2 >= dim[t2]) continue;
            for (int s1 = 0; s1 < 2; ++s1) {
                const int e1 = c[t1] - 1 + s1;
                if (e1 < 0 || e1 >= dim[t1]) continue;
                const int a1 = c[t1] - e1, a2 = c[t2] - e2;  // local coordinates of the node
                const double wq = 0.25 * h[t1] * h[t2];
                for (int q = 0; q < 4; ++q) {
                    const double xi1 = (q & 1) ? g1 : g0, xi2 = (q & 2) ? g1 : g0;
                    const double f1 = a1 ? xi1 : 1.0 - xi1, f2 = a2 ? xi2 : 1.0 - xi2;
                    const double N = f1 * f2;
                    // tangential gradient of the hat, dotted with k_hat
                    const double gk = (a1 ? 1.0 : -1.0) / h[t1] * f2 * wv.k[t1] +
                                      (a2 ? 1.0 : -1.0) / h[t2] * f1 * wv.k[t2];
                    double x[3];
                    x[nu] = org[nu] + (e_nu + side) * h[nu];
                    x[t1] = org[t1] + (e1 + xi1) * h[t1];
                    x[t2] = org[t2] + (e2 + xi2) * h[t2];
                    const double ph = -k0 * (wv.k[0] * x[0] + wv.k[1] * x[1] + wv.k[2] * x[2]);
                    double sn, cs;
                    sincos(ph, &sn, &cs);
                    // phase factor times amplitude
                    const double er = wv.ar * cs - wv.ai * sn, ei = wv.ar * sn + wv.ai * cs;
                    double hr[3], hi[3];
                    for (int d = 0; d < 3; ++d) {
                        hr[d] = wv.p[d] * er;
                        hi[d] = wv.p[d] * ei;
                    }
                    const double nhr = nsgn * hr[nu], nhi = nsgn * hi[nu];  // n . H_i
                    for (int al = 0; al < 3; ++al) {
                        // n x curl H_i = -j k0 (k_hat (n.H_i) - H_i (n.k_hat))
                        const double ur = wv.k[al] * nhr - hr[al] * nk, ui = wv.k[al] * nhi - hi[al] * nk;
                        // -N (n x curl H_i) = j k0 N u = k0 N (-ui + j ur)
                        double vr = -N * k0 * ui, vi = N * k0 * ur;
                        if (al != nu) {
                            // j k0 N H_al + sigma (j / 2k0)(grad_t N . (-j k0 k_t)) H_al
                            //   = j k0 N H_al + (sigma / 2)(grad_t N . k_hat) H_al
                            vr += -k0 * N * hi[al] + 0.5 * sigma * gk * hr[al];
                            vi += k0 * N * hr[al] + 0.5 * sigma * gk * hi[al];
                        }
                        br[al] += wq * vr;
                        bi[al] += wq * vi;
                    }
                }
            }
        }
    }
    // held by symmetry planes (and, for E, on conductor surfaces)
    unsigned fix = fixed_components(c[0], c[1], c[2], nx, ny, nz, planes);
    if (form_e) fix |= pec_held(mat, nx, ny, nz, c[0], c[1], c[2]);
    for (int al = 0; al < 3; ++al)
        B[((int64_t)3 * r + al) * nrhs + w] = (fix >> al) & 1u ? make_double2(0.0, 0.0) : make_double2(br[al], bi[al]);
}

fe_status build_rhs(fe_ctx* ctx, const fe_system* s, int nrhs, const fe_planewave* waves, double2* d_B,
                    DevBuf& wave_buf) {
    const fe_mesh* m = s->mesh;
    cudaStream_t st = ctx->stream;
    std::vector<Wave> hw(nrhs);
    for (int w = 0; w < nrhs; ++w) {
        for (int d = 0; d < 3; ++d) {
            hw[w].k[d] = waves[w].k_hat[d];
            hw[w].p[d] = waves[w].p_hat[d];
        }
        hw[w].ar = waves[w].amplitude.re;
        hw[w].ai = waves[w].amplitude.im;
    }
    FE_TRY(dev_alloc(st, wave_buf, (size_t)nrhs * sizeof(Wave)));
    FE_CUDA(cudaMemcpyAsync(wave_buf.ptr, hw.data(), (size_t)nrhs * sizeof(Wave), cudaMemcpyHostToDevice, st));
    const int64_t n = (int64_t)m->n_act * nrhs;
    k_rhs<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(m->nx, m->ny, m->nz, m->h[0], m->h[1], m->h[2],
                                                       m->origin[0], m->origin[1], m->origin[2], s->k0, s->sigma,
                                                       (const int*)m->node_id.ptr, m->n_act,
                                                       (const Wave*)wave_buf.ptr, nrhs, abc_faces(m->boundary),
                                                       pack_planes(m->boundary), (const uint8_t*)m->material.ptr,
                                                       s->formulation == FE_FORMULATION_E ? 1 : 0, d_B);
    FE_LAUNCHED();
    // the host staging vector must outlive the copy
    FE_CUDA(cudaStreamSynchronize(st));
    return FE_OK;
}

}  // namespace fe

using namespace fe;

extern "C" fe_status fe_rhs(fe_ctx* ctx, const fe_system* s, int32_t nrhs, const fe_planewave* waves, void* b_out,
                            int32_t on_device) {
    if (!ctx || !s || !waves || !b_out || nrhs < 1) {
        set_error("fe_rhs: NULL argument or nrhs < 1");
        return FE_ERR_INVALID_ARG;
    }
    cudaSetDevice(ctx->device);
    cudaStream_t st = ctx->stream;
    const size_t bytes = (size_t)3 * s->mesh->n_act * nrhs * sizeof(double2);
    DevBuf wb, tmp;
    double2* dB = (double2*)b_out;
    if (!on_device) {
        fe_status e = dev_alloc(st, tmp, bytes);
        if (e != FE_OK) return e;
        dB = (double2*)tmp.ptr;
    }
    fe_status e = build_rhs(ctx, s, nrhs, waves, dB, wb);
    if (e == FE_OK && !on_device) {
        cudaError_t ce = cudaMemcpyAsync(b_out, dB, bytes, cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) {
            set_error("fe_rhs copy: %s", cudaGetErrorString(ce));
            e = FE_ERR_CUDA;
        }
    }
    dev_free(st, wb);
    dev_free(st, tmp);
    return e;
}
