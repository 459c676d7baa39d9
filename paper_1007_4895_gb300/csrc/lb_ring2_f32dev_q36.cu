/* Layout-10 step kernel (the ring-fed step as a persistent kernel over row queues) for
 * one storage format and one high-order set size (one translation unit each, so that
 * they compile in parallel). */
#include "lb_ring2.cuh"

namespace lbk {
template void launch_ring_units_store<2, 36>(const StepParams<float> &, const RingTab &, const RowQueues &,
                                              int, void *);
template int launch_ring_batch_store<2, 36>(const StepParams<float> *, const RingTab *, const uint32_t *,
                                                 const int2 *, const int *, int, int, int, int, unsigned int *, bool,
                                                 int, int *, void *);
}

namespace lbk {
int ring_tab_build(const void *d_ctab, const StepParams<float> &p, RingTab *tab, void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PairTables *h = new PairTables;
    const bool ok = cudaMemcpyAsync(h, d_ctab, sizeof(PairTables), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                    cudaStreamSynchronize(st) == cudaSuccess;
    int rc = ok ? 0 : -1;
    auto sgn_f = [](float v) { return v > 0.0f ? 1 : (v < 0.0f ? -1 : 0); };
    auto sgn_i = [](int v) { return v > 0 ? 1 : (v < 0 ? -1 : 0); };
    for (int s = 0; s < 2 && rc == 0; ++s) {
        const int qs = p.set[s].q;
        const int n = qs == 9 ? 3 : (qs == 16 ? 4 : (qs == 36 ? 6 : 0));
        if (n == 0) rc = -1;
        for (int a = 0; a < LB_QMAX && rc == 0; ++a) {
            const PairC &pc = h->pp[s][a];
            const PairC2 &p2 = h->pp2[s][a];
            const MomC2 &pm = h->pm[s][a];
            if (a < qs && (sgn_f(pc.crx) != gh_sign(n, a % n) || sgn_i(pc.ystep) != gh_sign(n, a / n))) rc = -1;
            RingPop &r = tab->pop[s][a];
            r.cx2 = pc.cx2;
            r.cy2 = pc.cy2;
            r.ncx2 = pc.ncx2;
            r.nacy2 = pc.nacy2;
            r.ky2 = pc.ky2;
            r.gxi2 = p2.gxi2;
            r.w2 = p2.w2;
            r.winv2 = p2.winv2;
            r.wcx2 = pm.wcx2;
            r.wcy2 = pm.wcy2;
            r.kx = pc.kx;
            r.ystep = pc.ystep;
            const SetConst<float> &c = p.set[s];
            r.wxx = c.wxx[a];
            r.wxy = c.wxy[a];
            r.wyy = c.wyy[a];
            r.hxx = c.hxx[a];
            r.hxy = c.hxy[a];
            r.hyy = c.hyy[a];
        }
    }
    delete h;
    return rc;
}
}  // namespace lbk
