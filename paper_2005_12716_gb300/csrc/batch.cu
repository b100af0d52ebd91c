// Many independent sea states in one call (workload of uneven instances): every instance's
// reconstruction and gather are enqueued in order on one stream, so that a caller can capture
// one swense_batch_run call as a single CUDA graph and replay it as one launch. Scratch is the
// library workspace, which the first (uncaptured) call sizes for the largest instance.
#include "internal.cuh"

extern "C" int swense_batch_run(const swense_instance* inst, int32_t n, int32_t p_mode, double rho,
                                double g, void* stream) {
  if (n < 0) return swense::fail(SWENSE_ERR_ARG, "negative instance count");
  if (n > 0 && !inst) return swense::fail(SWENSE_ERR_ARG, "NULL instance array");
  for (int32_t i = 0; i < n; ++i) {
    const swense_instance& c = inst[i];
    int st = swense_fields_on_grid(&c.modes, c.n_tl, c.t_levels, &c.desc, c.nodes, c.eta, stream);
    if (st) return st;
    swense_grid gr{};
    gr.nodes = c.nodes;
    gr.eta = c.eta;
    gr.nx_r = c.desc.pad_n * c.modes.nx;
    gr.ny_r = c.modes.ny > 1 ? c.desc.pad_n * c.modes.ny : 1;
    gr.nz = c.desc.nz;
    gr.n_tl = c.n_tl;
    gr.Lx = c.modes.Lx;
    gr.Ly = c.modes.Ly;
    gr.z_levels = c.desc.z_levels;
    gr.t_levels = c.t_levels;
    gr.scheme = c.desc.scheme;
    st = c.perm ? swense_interp_permuted(&gr, c.t, c.pts, c.perm, c.np, c.out_eta, c.out_u, c.out_v,
                                         c.out_w, c.out_p, p_mode, rho, g, nullptr, stream)
                : swense_interp(&gr, c.t, c.pts, c.np, c.out_eta, c.out_u, c.out_v, c.out_w, c.out_p,
                                p_mode, rho, g, nullptr, stream);
    if (st) return st;
  }
  return SWENSE_OK;
}
