// api.cu -- the C ABI of include/ndt.h: context, device memory, host/device
// argument handling, exposure tables and launch sequencing.  All numerical
// work runs in the kernels of k_planes.cu, k_stack.cu and k_topk.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <limits>
#include <numeric>
#include <string>
#include <vector>

#include "ndt.h"
#include "ndt_internal.cuh"

using namespace ndt;

namespace {

// Grow-only device buffer owned by a context.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }   // every buffer of a context is freed with it
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) { p = nullptr; return e; }
    cap = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

char g_create_error[256] = "no error";

constexpr double kPi = 3.14159265358979323846;

}  // namespace

struct ndt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int n_sms = 0;
  std::string err = "no error";
  Phys ph{};
  double obliquity = 0.0;
  // exposures (sorted by epoch on the device)
  int32_t n_exp = 0;
  std::vector<ndt_exposure> table;
  std::vector<int32_t> sorted_to_table, table_to_sorted;
  std::vector<ExpDev> ex_host;
  int plane_type = kF32;
  DevBuf ex_dev, pos_to_table_dev, planes, jobs_dev, absmax_dev, plane_err;
  DevBuf stage_images, stage_vars;
  // orbit batch
  DevBuf stage_states, snr, out_tmp, xy_tmp;
  int64_t last_n = 0;
  // families and queue
  DevBuf fam_orb_off, fam_exp_off, fam_exp_pos, item_off, fam_order;
  DevBuf queue_head, counters;
  // top-k
  DevBuf topk_scratch, topk_out;
  // vetting
  DevBuf cand_stage, stamp_pos, stamp_f32, stamp_bf16, cnn_x, cnn_labels, cnn_out, cnn_scratch,
      cnn_params, cnn_grad, trim_bits, trim_nu, trim_n;
  // duplicate suppression
  DevBuf dedup_scratch, dedup_ref, dedup_out, count_dev;
  // noise estimate
  DevBuf mad_imgs, mad_state, mad_hist, mad_stage, mad_cnt, mad_buf;
  int64_t noise_bytes_read = 0;     // image bytes the last noise estimate streamed
  std::vector<float> noise_sigma;   // per exposure (table order): estimated sigma, or 0 if given
  // launch form
  int32_t mode = NDT_LAUNCH_PLAIN, orbit_tile = 64, exp_tile = 16, use_graph = 0;
  int32_t offchip = 1;     // off-chip test of the persistent form
  int32_t block_test = 1;  // warp cone test per exposure block (persistent form)
  int32_t geometry_fp64 = 0;  // plain form: FP64 light time and TAN projection
  int32_t state_df = 1;    // two-body state in double-float (both forms and predict_positions)
  int32_t footprint = 0;   // stack_orbits without families: walk orbits in sky-footprint order
  DevBuf fp_items, fp_hist;
  float broaden = 0.0f;    // filter broadening (px) for coarse searches
  double t_ref = 0.0;      // earliest exposure epoch (origin of ExpDev::tf)
  cudaGraphExec_t graph = nullptr;
  std::vector<unsigned char> graph_key;
  // stats
  int64_t launches = 0, samples = 0;
  cudaEvent_t ev[6] = {};
  bool have_stack_ev = false, have_planes_ev = false, have_topk_ev = false;
};

namespace {

ndt_status fail(ndt_ctx* c, ndt_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  c->err = buf;
  return s;
}

ndt_status cuda_fail(ndt_ctx* c, cudaError_t e, const char* what) {
  return fail(c, e == cudaErrorMemoryAllocation ? NDT_ENOMEM : NDT_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define NDT_CK(call, what)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Make `src` (host or device, `bytes` long) available on the device.
ndt_status to_device(ndt_ctx* ctx, const void* src, size_t bytes, DevBuf& stage, const void** out) {
  if (is_device_ptr(src)) {
    *out = src;
    return NDT_OK;
  }
  NDT_CK(stage.ensure(bytes), "staging allocation");
  NDT_CK(cudaMemcpyAsync(stage.p, src, bytes, cudaMemcpyHostToDevice, ctx->stream), "H2D copy");
  *out = stage.p;
  return NDT_OK;
}

void set_default_phys(ndt_ctx* c, double gm, double cl, double eps) {
  c->ph.gm = gm;
  c->ph.force_free = gm > 0.0 ? 0 : 1;
  c->ph.sqrt_gm = gm > 0.0 ? std::sqrt(gm) : 1.0;
  c->ph.inv_sqrt_gm = 1.0 / c->ph.sqrt_gm;
  c->ph.inv_gm = gm > 0.0 ? 1.0 / gm : 0.0;
  c->ph.inv_c = cl > 0.0 ? (float)(1.0 / cl) : 0.0f;
  c->ph.inv_c2 = cl > 0.0 ? (float)(1.0 / (cl * cl)) : 0.0f;
  {
    const dfloat g = split_df(gm > 0.0 ? gm : 0.0);
    c->ph.gm_f = g.h;
    c->ph.gm_l = g.l;
    const dfloat sg = split_df(c->ph.sqrt_gm), isg = split_df(c->ph.inv_sqrt_gm);
    c->ph.sgm_h = sg.h;
    c->ph.sgm_l = sg.l;
    c->ph.isgm_h = isg.h;
    c->ph.isgm_l = isg.l;
  }
  {
    const dfloat ic = split_df(cl > 0.0 ? 1.0 / cl : 0.0);
    c->ph.inv_c = ic.h;
    c->ph.inv_c_l = ic.l;
    c->ph.inv_c3 = cl > 0.0 ? (float)(1.0 / (cl * cl * cl)) : 0.0f;
  }
  c->obliquity = eps;
}

// Tangent-plane rows of one exposure in the ecliptic frame (TAN projection,
// Calabretta & Greisen 2002, sec. 5.1.3, with the inverse CD matrix folded in).
void derive_projection(const ndt_exposure& m, double eps, ExpDev& e) {
  const double d2r = kPi / 180.0;
  const double a0 = m.crval[0] * d2r, d0 = m.crval[1] * d2r;
  const double ca = std::cos(a0), sa = std::sin(a0), cdl = std::cos(d0), sdl = std::sin(d0);
  const double p0[3] = {cdl * ca, cdl * sa, sdl};
  const double ea[3] = {-sa, ca, 0.0};
  const double no[3] = {-sdl * ca, -sdl * sa, cdl};
  const double det = m.cd[0] * m.cd[3] - m.cd[1] * m.cd[2];
  const double i00 = m.cd[3] / det, i01 = -m.cd[1] / det, i10 = -m.cd[2] / det, i11 = m.cd[0] / det;
  const double r2d = 180.0 / kPi;
  double ax[3], ay[3];
  for (int i = 0; i < 3; ++i) {
    ax[i] = r2d * (i00 * ea[i] + i01 * no[i]);
    ay[i] = r2d * (i10 * ea[i] + i11 * no[i]);
  }
  // rows act on equatorial vectors q = R_x(eps) rho; fold R_x(eps)^T in
  const double ce = std::cos(eps), se = std::sin(eps);
  auto to_ecl = [&](const double w[3], double out[3]) {
    out[0] = w[0];
    out[1] = ce * w[1] + se * w[2];
    out[2] = -se * w[1] + ce * w[2];
  };
  to_ecl(p0, e.p0);
  to_ecl(ax, e.ax);
  to_ecl(ay, e.ay);
  e.crpix_h[0] = m.crpix[0] + 0.5;
  e.crpix_h[1] = m.crpix[1] + 0.5;
  // FP32 copies for the off-chip test; ppr = largest singular value of
  // CD^-1 (px/deg) in px/rad: the TAN map's stretch at the tangent point
  // (high parts by the device's own split, so both sides use one rounding)
  for (int i = 0; i < 3; ++i) {
    const dfloat p = split_df(e.p0[i]), a = split_df(e.ax[i]), b = split_df(e.ay[i]);
    e.p0_f[i] = p.h;
    e.p0_l[i] = p.l;
    e.ax_f[i] = a.h;
    e.ax_l[i] = a.l;
    e.ay_f[i] = b.h;
    e.ay_l[i] = b.l;
  }
  // rows with the reference pixel folded in (x + 1/2 = (rho . axc) / (rho . p0)),
  // summed in long double before the split
  for (int i = 0; i < 3; ++i) {
    const dfloat a = split_df((double)((long double)e.ax[i] + (long double)e.crpix_h[0] * e.p0[i]));
    const dfloat b = split_df((double)((long double)e.ay[i] + (long double)e.crpix_h[1] * e.p0[i]));
    e.axc_f[i] = a.h;
    e.axc_l[i] = a.l;
    e.ayc_f[i] = b.h;
    e.ayc_l[i] = b.l;
  }
  e.crpix_f[0] = (float)m.crpix[0];
  e.crpix_f[1] = (float)m.crpix[1];
  const double fro = i00 * i00 + i01 * i01 + i10 * i10 + i11 * i11, dt = i00 * i11 - i01 * i10;
  const double smax = std::sqrt(0.5 * (fro + std::sqrt(std::max(0.0, fro * fro - 4.0 * dt * dt))));
  e.ppr = (float)(smax * r2d * (1.0 + 1e-6));
  // largest off-axis angle of the chip: at a corner of [-1/2, W-1/2] x
  // [-1/2, H-1/2] (the TAN radius grows with the angle)
  double rmax = 0.0;
  for (int c = 0; c < 4; ++c) {
    const double px = (c & 1 ? m.width : 0) - 0.5 - m.crpix[0];
    const double py = (c & 2 ? m.height : 0) - 0.5 - m.crpix[1];
    const double xi = m.cd[0] * px + m.cd[1] * py, eta = m.cd[2] * px + m.cd[3] * py;   // deg
    rmax = std::max(rmax, std::sqrt(xi * xi + eta * eta) / r2d);
  }
  const double th = std::atan(rmax) + 0.01;
  e.cos_far = th < 0.5 * kPi ? (float)(std::cos(th) * (1.0 - 1e-6)) : -2.0f;
  // the chip cone of the block test: radius th (the corner angle + 0.01 rad)
  e.chip_cos = (float)std::cos(std::min(th, kPi));
  e.chip_sin = (float)std::sin(std::min(th, kPi));
}

// The power of two nearest to x > 0 (in log2), within the normal FP32 range.
float pow2_near(double x) {
  if (!(x > 0.0) || !std::isfinite(x)) return 1.0f;
  const int e = std::max(-120, std::min(120, (int)std::lround(std::log2(x))));
  return std::ldexp(1.0f, e);
}

// Sigma of the matched filter: the PSF's, broadened by the coarse-search
// smoothing when one is set (Gaussians convolve by adding variances).
float filter_sigma(const ndt_ctx* ctx, float psf_sigma) {
  if (ctx->broaden <= 0.0f) return psf_sigma;
  return (float)std::sqrt((double)psf_sigma * psf_sigma + (double)ctx->broaden * ctx->broaden);
}

void record(ndt_ctx* c, int i) { cudaEventRecord(c->ev[i], c->stream); }

// Iterative-MAD noise estimate of device images (k_mad.cu): (pass, pick)
// launches in groups of four until every image reaches its fixed point or
// max_rounds; a selection takes one to five passes, so 10 per round bound
// the loop.  out[i] is the final state of image i; the image bytes streamed
// are added to the context's statistics.
ndt_status mad_estimate(ndt_ctx* ctx, const std::vector<const float*>& dev_imgs,
                        const std::vector<int64_t>& n_pix, int max_rounds, std::vector<MadState>& out) {
  const int k = (int)dev_imgs.size();
  out.assign(k, mad_initial_state());
  ctx->noise_bytes_read = 0;
  if (k == 0) return NDT_OK;
  std::vector<MadImage> h(k);
  int64_t max_n = 0;
  for (int i = 0; i < k; ++i) {
    h[i] = MadImage{dev_imgs[i], n_pix[i]};
    max_n = std::max(max_n, n_pix[i]);
  }
  const uint32_t cap = (uint32_t)std::min<int64_t>(kMadCap, std::max<int64_t>(max_n, 1));
  NDT_CK(ctx->mad_imgs.ensure(sizeof(MadImage) * k), "noise image table");
  NDT_CK(ctx->mad_state.ensure(sizeof(MadState) * k), "noise state");
  NDT_CK(ctx->mad_hist.ensure(4 * mad_hist_words(k)), "noise histogram");
  NDT_CK(ctx->mad_cnt.ensure(4 * (size_t)k), "noise counters");
  NDT_CK(ctx->mad_buf.ensure(4 * (size_t)k * cap), "noise key buffer");
  NDT_CK(cudaMemcpyAsync(ctx->mad_imgs.p, h.data(), sizeof(MadImage) * k, cudaMemcpyHostToDevice, ctx->stream),
         "upload");
  NDT_CK(cudaMemcpyAsync(ctx->mad_state.p, out.data(), sizeof(MadState) * k, cudaMemcpyHostToDevice,
                         ctx->stream), "upload");
  NDT_CK(cudaMemsetAsync(ctx->mad_hist.p, 0, 4 * mad_hist_words(k), ctx->stream), "memset");
  NDT_CK(cudaMemsetAsync(ctx->mad_cnt.p, 0, 4 * (size_t)k, ctx->stream), "memset");
  constexpr int kGroup = 4;
  const int max_pairs = 10 * max_rounds + kGroup;
  for (int p = 0; p < max_pairs; p += kGroup) {
    NDT_CK(launch_mad_passes(ctx->mad_imgs.as<MadImage>(), ctx->mad_state.as<MadState>(),
                             ctx->mad_hist.as<uint32_t>(), ctx->mad_cnt.as<uint32_t>(),
                             ctx->mad_buf.as<uint32_t>(), cap, k, max_n, max_rounds, kGroup, ctx->stream),
           "noise kernels");
    ctx->launches += 2 * kGroup;
    NDT_CK(cudaMemcpyAsync(out.data(), ctx->mad_state.p, sizeof(MadState) * k, cudaMemcpyDeviceToHost,
                           ctx->stream), "state D2H");
    NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
    bool all = true;
    for (const MadState& st : out) all = all && st.done;
    if (all) break;
  }
  for (int i = 0; i < k; ++i) ctx->noise_bytes_read += (int64_t)out[i].passes * 4 * n_pix[i];
  return NDT_OK;
}

}  // namespace

extern "C" {

ndt_status ndt_create(ndt_ctx** out, int device, void* cuda_stream) {
  if (!out) return NDT_EINVAL;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || device < 0 || device >= ndev) {
    snprintf(g_create_error, sizeof g_create_error, "no CUDA device %d (%s)", device,
             e == cudaSuccess ? "out of range" : cudaGetErrorString(e));
    return e == cudaSuccess ? NDT_EINVAL : NDT_ECUDA;
  }
  e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    snprintf(g_create_error, sizeof g_create_error, "cudaSetDevice: %s", cudaGetErrorString(e));
    return NDT_ECUDA;
  }
  ndt_ctx* c = new ndt_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, device);
  set_default_phys(c, 0.01720209895 * 0.01720209895, 299792.458 * 86400.0 / 149597870.7,
                   84381.406 / 3600.0 * kPi / 180.0);
  for (auto& ev : c->ev) {
    if (cudaEventCreate(&ev) != cudaSuccess) {
      snprintf(g_create_error, sizeof g_create_error, "cudaEventCreate failed");
      delete c;
      return NDT_ECUDA;
    }
  }
  if (c->counters.ensure(64) != cudaSuccess || c->queue_head.ensure(64) != cudaSuccess) {
    snprintf(g_create_error, sizeof g_create_error, "device allocation failed");
    delete c;
    return NDT_ENOMEM;
  }
  cudaMemset(c->counters.p, 0, 64);
  *out = c;
  return NDT_OK;
}

void ndt_destroy(ndt_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (auto& ev : c->ev)
    if (ev) cudaEventDestroy(ev);
  DevBuf* bufs[] = {&c->ex_dev, &c->pos_to_table_dev, &c->planes, &c->jobs_dev,
                    &c->absmax_dev, &c->plane_err, &c->stage_images, &c->stage_vars,
                    &c->stage_states, &c->snr, &c->out_tmp, &c->xy_tmp, &c->fam_orb_off,
                    &c->fam_exp_off, &c->fam_exp_pos, &c->item_off, &c->fam_order,
                    &c->queue_head, &c->counters, &c->topk_scratch, &c->topk_out,
                    &c->cand_stage, &c->stamp_pos, &c->stamp_f32, &c->stamp_bf16, &c->cnn_x,
                    &c->cnn_labels, &c->cnn_out, &c->cnn_scratch, &c->cnn_params, &c->cnn_grad,
                    &c->dedup_scratch, &c->dedup_ref, &c->dedup_out, &c->count_dev,
                    &c->trim_bits, &c->trim_nu, &c->trim_n, &c->mad_imgs, &c->mad_state,
                    &c->mad_hist, &c->mad_stage, &c->mad_cnt, &c->mad_buf, &c->fp_items, &c->fp_hist};
  for (DevBuf* b : bufs) b->release();
  delete c;   // (the DevBuf destructors free anything not listed above)
}

const char* ndt_last_error(const ndt_ctx* c) { return c ? c->err.c_str() : g_create_error; }

ndt_status ndt_set_constants(ndt_ctx* ctx, double gm, double c_light, double obliquity_rad) {
  if (!ctx) return NDT_EINVAL;
  if (!std::isfinite(gm) || !std::isfinite(c_light) || !std::isfinite(obliquity_rad))
    return fail(ctx, NDT_EINVAL, "constants must be finite");
  set_default_phys(ctx, gm, c_light, obliquity_rad);
  if (ctx->n_exp > 0) {   // the projection rows depend on the obliquity
    for (int s = 0; s < ctx->n_exp; ++s)
      derive_projection(ctx->table[ctx->sorted_to_table[s]], ctx->obliquity, ctx->ex_host[s]);
    NDT_CK(cudaMemcpyAsync(ctx->ex_dev.p, ctx->ex_host.data(), sizeof(ExpDev) * ctx->n_exp,
                           cudaMemcpyHostToDevice, ctx->stream), "exposure upload");
    NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  }
  return NDT_OK;
}

ndt_status ndt_load_exposures(ndt_ctx* ctx, const ndt_exposure* meta, int32_t n_exp,
                              const float* const* images, const float* const* variances,
                              int32_t plane_dtype) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (!meta || !images || n_exp < 1 || n_exp > 65535)
    return fail(ctx, NDT_EINVAL, "meta/images null or n_exp outside [1, 65535]");
  if (plane_dtype < 0 || plane_dtype > 2) return fail(ctx, NDT_EINVAL, "bad plane dtype %d", plane_dtype);
  for (int j = 0; j < n_exp; ++j) {
    const ndt_exposure& m = meta[j];
    const double det = m.cd[0] * m.cd[3] - m.cd[1] * m.cd[2];
    if (!images[j]) return fail(ctx, NDT_EINVAL, "image %d is null", j);
    if (!std::isfinite(m.mjd)) return fail(ctx, NDT_EINVAL, "exposure %d: epoch not finite", j);
    if (!(m.psf_sigma_px > 0.0f && m.psf_sigma_px <= 4.0f))
      return fail(ctx, NDT_EINVAL, "exposure %d: psf sigma %g outside (0, 4]", j, m.psf_sigma_px);
    if (!(filter_sigma(ctx, m.psf_sigma_px) <= 4.0f))
      return fail(ctx, NDT_EINVAL, "exposure %d: broadened filter sigma %g above 4 px", j,
                  filter_sigma(ctx, m.psf_sigma_px));
    if (!variances && std::isnan(m.variance))
      return fail(ctx, NDT_EINVAL, "exposure %d: variance is NaN", j);
    if (!(std::isfinite(det) && det != 0.0)) return fail(ctx, NDT_EINVAL, "exposure %d: singular CD", j);
    if (m.width < 1 || m.height < 1 || m.width > 32768 || m.height > 32768)
      return fail(ctx, NDT_EINVAL, "exposure %d: size %dx%d", j, m.width, m.height);
    if (variances && !variances[j]) return fail(ctx, NDT_EINVAL, "variance plane %d is null", j);
  }
  ctx->n_exp = 0;
  ctx->table.assign(meta, meta + n_exp);
  ctx->sorted_to_table.resize(n_exp);
  std::iota(ctx->sorted_to_table.begin(), ctx->sorted_to_table.end(), 0);
  std::stable_sort(ctx->sorted_to_table.begin(), ctx->sorted_to_table.end(),
                   [&](int a, int b) { return meta[a].mjd < meta[b].mjd; });
  ctx->table_to_sorted.assign(n_exp, 0);
  for (int s = 0; s < n_exp; ++s) ctx->table_to_sorted[ctx->sorted_to_table[s]] = s;
  ctx->t_ref = meta[ctx->sorted_to_table[0]].mjd;

  // plane layout (sorted order), staging of host images
  ctx->ex_host.assign(n_exp, ExpDev{});
  std::vector<PlaneJob> jobs(n_exp);
  std::vector<double> sum_p2(n_exp);   // sum of P^2 over the PSF window
  int64_t plane_elems = 0, img_elems = 0;
  for (int s = 0; s < n_exp; ++s) {
    const ndt_exposure& m = meta[ctx->sorted_to_table[s]];
    ExpDev& e = ctx->ex_host[s];
    e.t = m.mjd;
    for (int i = 0; i < 3; ++i) e.obs[i] = m.obs_xyz[i];
    derive_projection(m, ctx->obliquity, e);
    {
      const dfloat tt = split_df(m.mjd - ctx->t_ref);
      e.tf = tt.h;
      e.tf_l = tt.l;
    }
    for (int i = 0; i < 3; ++i) {
      const dfloat o = split_df(m.obs_xyz[i]);
      e.obs_f[i] = o.h;
      e.obs_l[i] = o.l;
    }
    e.W = m.width;
    e.H = m.height;
    e.tiles_x = (m.width + kTile - 1) / kTile;
    const int tiles_y = (m.height + kTile - 1) / kTile;
    e.plane_off = plane_elems;
    e.s_psi = 1.0f;
    e.s_phi = 1.0f;
    plane_elems += (int64_t)e.tiles_x * tiles_y * kTile * kTile;
    PlaneJob& J = jobs[s];
    J.var_c = m.variance > 0.0f ? m.variance : 1.0f;
    J.sigma = filter_sigma(ctx, m.psf_sigma_px);
    // unit-sum 1-D Gaussian window of the truncated PSF (FP64, rounded once)
    J.R = (int)std::ceil(4.0 * (double)J.sigma);
    {
      double w[2 * kMaxPsfRadius + 1], sum = 0.0;
      const double s2 = 2.0 * (double)J.sigma * (double)J.sigma;
      for (int k = -J.R; k <= J.R; ++k) sum += (w[k + J.R] = std::exp(-(double)(k * k) / s2));
      double sg2 = 0.0;
      for (int k = 0; k <= 2 * J.R; ++k) {
        const double g = w[k] / sum;
        J.g[k] = (float)g;
        J.g2[k] = (float)(g * g);
        sg2 += g * g;
      }
      // BF16 scales: the noise sigma of psi, sqrt(sum P^2 / V), and the
      // interior value of phi, sum P^2 / V (sum P^2 = (sum g^2)^2), each
      // rounded to a power of two (BF16 has the FP32 exponent range, so the
      // scale only centres the values; a power of two makes the division by
      // it an exact multiplication in the planes kernel and the gather)
      const double vbar = variances ? 1.0 : (double)J.var_c;
      J.s_phi = pow2_near(sg2 * sg2 / vbar);
      J.s_psi = pow2_near(std::sqrt(sg2 * sg2 / vbar));
      sum_p2[s] = sg2 * sg2;
    }
    J.W = m.width;
    J.H = m.height;
    J.tiles_x = e.tiles_x;
    J.tiles_y = tiles_y;
    J.plane_off = e.plane_off;
    img_elems += (int64_t)m.width * m.height;
  }
  // images: device pointers are used in place, host images are staged
  bool any_host_img = false, any_host_var = false;
  for (int j = 0; j < n_exp; ++j) {
    if (!is_device_ptr(images[j])) any_host_img = true;
    if (variances && !is_device_ptr(variances[j])) any_host_var = true;
  }
  if (any_host_img) NDT_CK(ctx->stage_images.ensure(sizeof(float) * img_elems), "image staging");
  if (any_host_var) NDT_CK(ctx->stage_vars.ensure(sizeof(float) * img_elems), "variance staging");
  int64_t img_off = 0;
  // host images that follow each other in memory (in epoch order) go over in
  // one copy: a run [run_src, run_src + run_bytes) to run_dst
  const char* run_src = nullptr;
  char* run_dst = nullptr;
  size_t run_bytes = 0;
  auto flush_run = [&]() -> cudaError_t {
    cudaError_t e = cudaSuccess;
    if (run_bytes) e = cudaMemcpyAsync(run_dst, run_src, run_bytes, cudaMemcpyHostToDevice, ctx->stream);
    run_bytes = 0;
    return e;
  };
  for (int s = 0; s < n_exp; ++s) {
    const int j = ctx->sorted_to_table[s];
    const size_t bytes = sizeof(float) * (size_t)meta[j].width * meta[j].height;
    PlaneJob& J = jobs[s];
    if (is_device_ptr(images[j])) {
      J.image = images[j];
    } else {
      float* dst = ctx->stage_images.as<float>() + img_off;
      const char* src = reinterpret_cast<const char*>(images[j]);
      if (!(run_bytes && src == run_src + run_bytes && reinterpret_cast<char*>(dst) == run_dst + run_bytes)) {
        NDT_CK(flush_run(), "image H2D");
        run_src = src;
        run_dst = reinterpret_cast<char*>(dst);
      }
      run_bytes += bytes;
      J.image = dst;
    }
    J.var = nullptr;
    if (variances) {
      if (is_device_ptr(variances[j])) {
        J.var = variances[j];
      } else {
        float* dst = ctx->stage_vars.as<float>() + img_off;
        NDT_CK(cudaMemcpyAsync(dst, variances[j], bytes, cudaMemcpyHostToDevice, ctx->stream),
               "variance H2D");
        J.var = dst;
      }
    }
    img_off += (int64_t)meta[j].width * meta[j].height;
  }
  NDT_CK(flush_run(), "image H2D");
  // exposures without a variance (<= 0, no variance planes): iterative MAD
  ctx->noise_sigma.assign(n_exp, 0.0f);
  if (!variances) {
    std::vector<const float*> imgs;
    std::vector<int64_t> npx;
    std::vector<int> which;
    for (int s = 0; s < n_exp; ++s) {
      const ndt_exposure& m = meta[ctx->sorted_to_table[s]];
      if (m.variance > 0.0f) continue;
      imgs.push_back(jobs[s].image);
      npx.push_back((int64_t)m.width * m.height);
      which.push_back(s);
    }
    std::vector<MadState> est;
    ndt_status st = mad_estimate(ctx, imgs, npx, kNoiseMaxRounds, est);
    if (st != NDT_OK) return st;
    for (size_t i = 0; i < which.size(); ++i) {
      const int s = which[i];
      const float sg = est[i].sigma;
      if (!(sg > 0.0f) || !std::isfinite(sg))
        return fail(ctx, NDT_EINVAL, "exposure %d: noise estimate %g is not positive",
                    ctx->sorted_to_table[s], sg);
      PlaneJob& J = jobs[s];
      J.var_c = (float)((double)sg * (double)sg);
      J.s_phi = pow2_near(sum_p2[s] / (double)J.var_c);
      J.s_psi = pow2_near(std::sqrt(sum_p2[s] / (double)J.var_c));
      ctx->noise_sigma[ctx->sorted_to_table[s]] = sg;
    }
  }
  int max_R = 0;
  for (const PlaneJob& J : jobs) max_R = std::max(max_R, J.R);
  plane_jobs_prepare(jobs.data(), n_exp, max_R);
  NDT_CK(ctx->jobs_dev.ensure(sizeof(PlaneJob) * n_exp), "job table");
  NDT_CK(cudaMemcpyAsync(ctx->jobs_dev.p, jobs.data(), sizeof(PlaneJob) * n_exp,
                         cudaMemcpyHostToDevice, ctx->stream), "job upload");
  NDT_CK(ctx->plane_err.ensure(4), "plane error word");
  NDT_CK(cudaMemsetAsync(ctx->plane_err.p, 0, 4, ctx->stream), "memset");
  unsigned int* perr = ctx->plane_err.as<unsigned int>();
  const bool any_var = variances != nullptr;
  const size_t pair_bytes = plane_dtype == NDT_PLANE_F32 ? 8 : 4;
  NDT_CK(ctx->planes.ensure(pair_bytes * plane_elems), "plane allocation");
  record(ctx, 0);
  if (plane_dtype == NDT_PLANE_F32) {
    NDT_CK(launch_planes(ctx->jobs_dev.as<PlaneJob>(), jobs.data(), n_exp, max_R, any_var, kPlaneStoreF32,
                         ctx->planes.p, nullptr, perr, ctx->stream), "plane kernel");
    ctx->launches += 1;
  } else if (plane_dtype == NDT_PLANE_BF16) {
    NDT_CK(launch_planes(ctx->jobs_dev.as<PlaneJob>(), jobs.data(), n_exp, max_R, any_var,
                         kPlaneStoreBF16, ctx->planes.p, nullptr, perr, ctx->stream), "plane kernel");
    ctx->launches += 1;
    for (int s = 0; s < n_exp; ++s) {
      ctx->ex_host[s].s_psi = jobs[s].s_psi;
      ctx->ex_host[s].s_phi = jobs[s].s_phi;
    }
  } else {
    // pass 1: largest |psi| and phi per plane (nothing stored); pass 2: the
    // same planes again, written as FP16 pairs scaled by those maxima
    NDT_CK(ctx->absmax_dev.ensure(8 * n_exp), "absmax");
    NDT_CK(cudaMemsetAsync(ctx->absmax_dev.p, 0, 8 * n_exp, ctx->stream), "memset");
    NDT_CK(launch_planes(ctx->jobs_dev.as<PlaneJob>(), jobs.data(), n_exp, max_R, any_var, kPlaneAbsMax,
                         nullptr, ctx->absmax_dev.as<unsigned int>(), perr, ctx->stream),
           "plane max kernel");
    NDT_CK(launch_planes(ctx->jobs_dev.as<PlaneJob>(), jobs.data(), n_exp, max_R, any_var,
                         kPlaneStoreF16,
                         ctx->planes.p, ctx->absmax_dev.as<unsigned int>(), perr, ctx->stream),
           "plane kernel");
    ctx->launches += 2;
  }
  record(ctx, 1);
  ctx->have_planes_ev = true;
  if (plane_dtype == NDT_PLANE_F16) {
    std::vector<unsigned int> mx(2 * n_exp);
    NDT_CK(cudaMemcpyAsync(mx.data(), ctx->absmax_dev.p, 8 * n_exp, cudaMemcpyDeviceToHost,
                           ctx->stream), "scale read-back");
    NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
    for (int s = 0; s < n_exp; ++s) {   // the kernel's scales: max / 2^14, or 1 for an empty plane
      float a0, a1;
      std::memcpy(&a0, &mx[2 * s], 4);
      std::memcpy(&a1, &mx[2 * s + 1], 4);
      ctx->ex_host[s].s_psi = a0 > 0.0f ? a0 / 16384.0f : 1.0f;
      ctx->ex_host[s].s_phi = a1 > 0.0f ? a1 / 16384.0f : 1.0f;
    }
  }
  NDT_CK(ctx->ex_dev.ensure(sizeof(ExpDev) * n_exp), "exposure table");
  NDT_CK(cudaMemcpyAsync(ctx->ex_dev.p, ctx->ex_host.data(), sizeof(ExpDev) * n_exp,
                         cudaMemcpyHostToDevice, ctx->stream), "exposure upload");
  NDT_CK(ctx->pos_to_table_dev.ensure(4 * n_exp), "permutation");
  NDT_CK(cudaMemcpyAsync(ctx->pos_to_table_dev.p, ctx->sorted_to_table.data(), 4 * n_exp,
                         cudaMemcpyHostToDevice, ctx->stream), "permutation upload");
  unsigned int plane_err_h = 0;
  NDT_CK(cudaMemcpyAsync(&plane_err_h, perr, 4, cudaMemcpyDeviceToHost, ctx->stream), "error read-back");
  // host vectors above must outlive the async copies
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  if (plane_err_h != 0)
    return fail(ctx, NDT_ETIMEOUT, "planes kernel: %u TMA loads did not arrive within the wait limit",
                plane_err_h);
  ctx->plane_type = plane_dtype;
  ctx->n_exp = n_exp;
  ctx->last_n = 0;
  return NDT_OK;
}

}  // extern "C"

namespace {

// Families on the host: validate, map exposures to sorted positions (epoch
// order within each family), build the queue order (families with more
// exposures first) and upload.
ndt_status prepare_families(ndt_ctx* ctx, int64_t n, const int64_t* fo_in, const int64_t* fe_in,
                            const int32_t* fi_in, int32_t n_fam, bool need_queue, int team,
                            StackArgs& a) {
  std::vector<int64_t> fo, fe;
  std::vector<int32_t> fi;
  if (n_fam > 0) {
    if (!fo_in || !fe_in || !fi_in) return fail(ctx, NDT_EINVAL, "family arrays must be non-null");
    fo.resize(n_fam + 1);
    fe.resize(n_fam + 1);
    auto fetch = [&](const void* src, void* dst, size_t bytes) -> cudaError_t {
      if (is_device_ptr(src)) return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
      std::memcpy(dst, src, bytes);
      return cudaSuccess;
    };
    NDT_CK(fetch(fo_in, fo.data(), 8 * (n_fam + 1)), "family offsets");
    NDT_CK(fetch(fe_in, fe.data(), 8 * (n_fam + 1)), "family exposure offsets");
    if (fo[0] != 0 || fo[n_fam] != n) return fail(ctx, NDT_EINVAL, "family orbit offsets must span [0, n)");
    if (fe[0] != 0) return fail(ctx, NDT_EINVAL, "family exposure offsets must start at 0");
    for (int f = 0; f < n_fam; ++f)
      if (fo[f + 1] < fo[f] || fe[f + 1] < fe[f]) return fail(ctx, NDT_EINVAL, "offsets decrease at %d", f);
    fi.resize(fe[n_fam]);
    if (!fi.empty()) NDT_CK(fetch(fi_in, fi.data(), 4 * fi.size()), "family exposure list");
    std::vector<unsigned char> seen(ctx->n_exp, 0);
    for (int f = 0; f < n_fam; ++f) {
      for (int64_t k = fe[f]; k < fe[f + 1]; ++k) {
        const int32_t j = fi[k];
        if (j < 0 || j >= ctx->n_exp) return fail(ctx, NDT_EINVAL, "family %d: exposure %d out of range", f, j);
        if (seen[j]) return fail(ctx, NDT_EINVAL, "family %d: exposure %d repeated", f, j);
        seen[j] = 1;
        fi[k] = ctx->table_to_sorted[j];
      }
      for (int64_t k = fe[f]; k < fe[f + 1]; ++k) seen[ctx->sorted_to_table[fi[k]]] = 0;
      std::sort(fi.begin() + fe[f], fi.begin() + fe[f + 1]);
    }
  } else if (need_queue) {
    n_fam = 1;
    fo = {0, n};
    fe = {0, (int64_t)ctx->n_exp};
    fi.resize(ctx->n_exp);
    std::iota(fi.begin(), fi.end(), 0);
  }
  a.n_fam = n_fam;
  a.fam_orb_off = a.fam_exp_off = nullptr;
  a.fam_exp_pos = nullptr;
  a.item_off = nullptr;
  a.fam_order = nullptr;
  a.n_items = 0;
  ctx->samples = 0;
  if (n_fam == 0) {
    ctx->samples = n * (int64_t)ctx->n_exp;
    return NDT_OK;
  }
  for (int f = 0; f < n_fam; ++f) ctx->samples += (fo[f + 1] - fo[f]) * (fe[f + 1] - fe[f]);
  NDT_CK(ctx->fam_orb_off.ensure(8 * (n_fam + 1)), "family buffers");
  NDT_CK(ctx->fam_exp_off.ensure(8 * (n_fam + 1)), "family buffers");
  NDT_CK(ctx->fam_exp_pos.ensure(4 * std::max<size_t>(fi.size(), 1)), "family buffers");
  NDT_CK(cudaMemcpyAsync(ctx->fam_orb_off.p, fo.data(), 8 * (n_fam + 1), cudaMemcpyHostToDevice, ctx->stream), "upload");
  NDT_CK(cudaMemcpyAsync(ctx->fam_exp_off.p, fe.data(), 8 * (n_fam + 1), cudaMemcpyHostToDevice, ctx->stream), "upload");
  if (!fi.empty())
    NDT_CK(cudaMemcpyAsync(ctx->fam_exp_pos.p, fi.data(), 4 * fi.size(), cudaMemcpyHostToDevice, ctx->stream), "upload");
  a.fam_orb_off = ctx->fam_orb_off.as<int64_t>();
  a.fam_exp_off = ctx->fam_exp_off.as<int64_t>();
  a.fam_exp_pos = ctx->fam_exp_pos.as<int32_t>();
  std::vector<int64_t> item_off;
  std::vector<int32_t> order;
  if (need_queue) {
    order.resize(n_fam);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      return (fe[x + 1] - fe[x]) > (fe[y + 1] - fe[y]);
    });
    item_off.resize(n_fam + 1);
    item_off[0] = 0;
    for (int q = 0; q < n_fam; ++q) {
      const int f = order[q];
      item_off[q + 1] = item_off[q] + (fo[f + 1] - fo[f] + team - 1) / team;
    }
    NDT_CK(ctx->item_off.ensure(8 * (n_fam + 1)), "queue buffers");
    NDT_CK(ctx->fam_order.ensure(4 * n_fam), "queue buffers");
    NDT_CK(cudaMemcpyAsync(ctx->item_off.p, item_off.data(), 8 * (n_fam + 1), cudaMemcpyHostToDevice, ctx->stream), "upload");
    NDT_CK(cudaMemcpyAsync(ctx->fam_order.p, order.data(), 4 * n_fam, cudaMemcpyHostToDevice, ctx->stream), "upload");
    a.item_off = ctx->item_off.as<int64_t>();
    a.fam_order = ctx->fam_order.as<int32_t>();
    a.n_items = item_off[n_fam];
  }
  // the host vectors are released on return: wait for their uploads
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  return NDT_OK;
}

ndt_status run_stack(ndt_ctx* ctx, StackArgs& a) {
  if (ctx->mode == NDT_LAUNCH_PLAIN) {
    NDT_CK(cudaMemsetAsync(ctx->counters.p, 0, 16, ctx->stream), "memset");
    NDT_CK(cudaMemsetAsync(ctx->counters.as<unsigned long long>() + 3, 0, 16, ctx->stream), "memset");
    record(ctx, 2);
    NDT_CK(launch_stack_plain(a, ctx->stream), "stack kernel");
    record(ctx, 3);
    ctx->launches += 1;
    ctx->have_stack_ev = true;
    return NDT_OK;
  }
  a.queue_head = ctx->queue_head.as<unsigned long long>();
  auto enqueue = [&]() -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(ctx->queue_head.p, 0, 8, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->counters.p, 0, 16, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->counters.as<unsigned long long>() + 3, 0, 16, ctx->stream);
    if (e == cudaSuccess) e = launch_stack_persistent(a, ctx->n_sms, ctx->stream);
    return e;
  };
  if (ctx->use_graph) {
    std::vector<unsigned char> key(sizeof(StackArgs) + 8);
    std::memcpy(key.data(), &a, sizeof(StackArgs));
    const int64_t extra = ((int64_t)ctx->orbit_tile << 32) | ctx->exp_tile;
    std::memcpy(key.data() + sizeof(StackArgs), &extra, 8);
    if (!ctx->graph || key != ctx->graph_key) {
      if (ctx->graph) { cudaGraphExecDestroy(ctx->graph); ctx->graph = nullptr; }
      cudaGraph_t g;
      NDT_CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "capture begin");
      cudaError_t e = enqueue();
      cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
      if (e != cudaSuccess) {
        if (e2 == cudaSuccess) cudaGraphDestroy(g);
        return cuda_fail(ctx, e, "captured stack");
      }
      NDT_CK(e2, "capture end");
      NDT_CK(cudaGraphInstantiate(&ctx->graph, g, 0), "graph instantiate");
      cudaGraphDestroy(g);
      ctx->graph_key = key;
    }
    record(ctx, 2);
    NDT_CK(cudaGraphLaunch(ctx->graph, ctx->stream), "graph launch");
    record(ctx, 3);
  } else {
    record(ctx, 2);
    NDT_CK(enqueue(), "persistent stack");
    record(ctx, 3);
  }
  ctx->launches += 1;
  ctx->have_stack_ev = true;
  return NDT_OK;
}

}  // namespace

extern "C" {

ndt_status ndt_stack_orbits(ndt_ctx* ctx, const double* states, double t0, int64_t n_orbits,
                            const int64_t* fam_orbit_off, const int64_t* fam_exp_off,
                            const int32_t* fam_exp_idx, int32_t n_fam, int32_t min_obs,
                            float* psi_sum, float* phi_sum, int32_t* nobs, float* snr) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (ctx->n_exp < 1) return fail(ctx, NDT_ESTATE, "stack_orbits before load_exposures");
  if (n_orbits < 0 || n_orbits > 0xffffffffll) return fail(ctx, NDT_EINVAL, "n_orbits %lld out of range", (long long)n_orbits);
  if (n_orbits > 0 && !states) return fail(ctx, NDT_EINVAL, "states is null");
  if (n_fam < 0) return fail(ctx, NDT_EINVAL, "n_fam < 0");
  if (!std::isfinite(t0)) return fail(ctx, NDT_EINVAL, "t0 not finite");
  // zeroed bytes, padding included: the graph-reuse key compares the raw bytes
  StackArgs a;
  std::memset(&a, 0, sizeof a);
  const bool persistent = ctx->mode == NDT_LAUNCH_PERSISTENT;
  ndt_status s = prepare_families(ctx, n_orbits, fam_orbit_off, fam_exp_off, fam_exp_idx, n_fam,
                                  persistent, ctx->orbit_tile, a);
  if (s != NDT_OK) return s;
  ctx->last_n = 0;
  if (n_orbits == 0) return NDT_OK;
  const void* st_dev = nullptr;
  s = to_device(ctx, states, sizeof(double) * 6 * n_orbits, ctx->stage_states, &st_dev);
  if (s != NDT_OK) return s;
  NDT_CK(ctx->snr.ensure(4 * n_orbits), "snr buffer");
  // host outputs go through a device scratch of 3 arrays
  const bool h_psi = psi_sum && !is_device_ptr(psi_sum), h_phi = phi_sum && !is_device_ptr(phi_sum);
  const bool h_nobs = nobs && !is_device_ptr(nobs), h_snr = snr && !is_device_ptr(snr);
  if (h_psi || h_phi || h_nobs) NDT_CK(ctx->out_tmp.ensure(12 * n_orbits), "output scratch");
  a.states = static_cast<const double*>(st_dev);
  a.n = n_orbits;
  a.t0 = t0;
  a.ex = ctx->ex_dev.as<ExpDev>();
  a.n_exp = ctx->n_exp;
  a.planes = ctx->planes.p;
  a.plane_type = ctx->plane_type;
  a.orbit_tile = ctx->orbit_tile;
  a.exp_tile = ctx->exp_tile;
  a.psi_sum = h_psi ? ctx->out_tmp.as<float>() : psi_sum;
  a.phi_sum = h_phi ? ctx->out_tmp.as<float>() + n_orbits : phi_sum;
  a.nobs = h_nobs ? reinterpret_cast<int32_t*>(ctx->out_tmp.as<float>() + 2 * n_orbits) : nobs;
  a.snr = ctx->snr.as<float>();
  a.min_obs = min_obs;
  a.counters = ctx->counters.as<unsigned long long>();
  a.ph = ctx->ph;
  a.t_ref = ctx->t_ref;
  a.offchip_test = persistent ? ctx->offchip : 0;
  a.block_test = persistent && ctx->offchip ? ctx->block_test : 0;
  a.geometry_fp64 = persistent ? 0 : ctx->geometry_fp64;
  a.state_df = ctx->state_df;
  if (ctx->footprint && n_fam == 0 && n_orbits > 1) {
    // orbits ordered by their sky direction at the middle exposure, so that
    // a warp's orbits gather from the same image tiles and the off-chip and
    // block tests can skip whole warps; outputs stay in the caller's order
    NDT_CK(ctx->fp_items.ensure(16 * (size_t)n_orbits), "footprint keys");
    NDT_CK(ctx->fp_hist.ensure(sort_hist_bytes(n_orbits)), "footprint histogram");
    unsigned long long* ia = ctx->fp_items.as<unsigned long long>();
    unsigned long long* sorted = nullptr;
    NDT_CK(launch_footprint_order(a.states, n_orbits, t0, ctx->t_ref, a.ex, ctx->n_exp / 2, ctx->ph,
                                  ctx->state_df != 0, ia, ia + n_orbits, ctx->fp_hist.as<unsigned int>(), &sorted,
                                  ctx->stream),
           "footprint order");
    ctx->launches += 13;
    a.order = sorted;
  }
  s = run_stack(ctx, a);
  if (s != NDT_OK) return s;
  ctx->last_n = n_orbits;
  if (snr && !h_snr)
    NDT_CK(cudaMemcpyAsync(snr, ctx->snr.p, 4 * n_orbits, cudaMemcpyDeviceToDevice, ctx->stream), "snr copy");
  if (h_psi || h_phi || h_nobs || h_snr) {
    if (h_psi) NDT_CK(cudaMemcpyAsync(psi_sum, a.psi_sum, 4 * n_orbits, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
    if (h_phi) NDT_CK(cudaMemcpyAsync(phi_sum, a.phi_sum, 4 * n_orbits, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
    if (h_nobs) NDT_CK(cudaMemcpyAsync(nobs, a.nobs, 4 * n_orbits, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
    if (h_snr) NDT_CK(cudaMemcpyAsync(snr, ctx->snr.p, 4 * n_orbits, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
    NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
    unsigned long long cnt[2];
    NDT_CK(cudaMemcpy(cnt, ctx->counters.p, 16, cudaMemcpyDeviceToHost), "counters");
    if (cnt[1]) return fail(ctx, NDT_ENOCONV, "%llu Kepler solves did not converge", cnt[1]);
  }
  return NDT_OK;
}

ndt_status ndt_topk_candidates(ndt_ctx* ctx, int64_t k, int64_t* idx_out, float* snr_out,
                               int64_t* k_out) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (ctx->last_n <= 0) return fail(ctx, NDT_ESTATE, "topk_candidates without a stacked batch");
  if (k < 0) return fail(ctx, NDT_EINVAL, "k < 0");
  const int64_t n = ctx->last_n;
  if (k > n) k = n;
  if (k_out) *k_out = k;
  if (k == 0) return NDT_OK;
  const size_t sb = topk_scratch_bytes(n, k);
  NDT_CK(ctx->topk_scratch.ensure(sb), "top-k scratch");
  const bool h_idx = idx_out && !is_device_ptr(idx_out), h_snr = snr_out && !is_device_ptr(snr_out);
  if (h_idx || h_snr) NDT_CK(ctx->topk_out.ensure(12 * k), "top-k output scratch");
  int64_t* di = h_idx ? ctx->topk_out.as<int64_t>() : idx_out;
  float* ds = h_snr ? reinterpret_cast<float*>(ctx->topk_out.as<int64_t>() + k) : snr_out;
  int L = 0;
  record(ctx, 4);
  NDT_CK(launch_topk(ctx->snr.as<float>(), n, k, ctx->topk_scratch.p, ctx->topk_scratch.cap, di, ds,
                     &L, ctx->stream), "top-k kernels");
  record(ctx, 5);
  ctx->have_topk_ev = true;
  ctx->launches += L;
  if (h_idx) NDT_CK(cudaMemcpyAsync(idx_out, di, 8 * k, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  if (h_snr) NDT_CK(cudaMemcpyAsync(snr_out, ds, 4 * k, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  return NDT_OK;
}

ndt_status ndt_count_candidates(ndt_ctx* ctx, float min_snr, int64_t* count) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (ctx->last_n <= 0) return fail(ctx, NDT_ESTATE, "count_candidates without a stacked batch");
  if (!count || std::isnan(min_snr)) return fail(ctx, NDT_EINVAL, "bad count arguments");
  NDT_CK(ctx->count_dev.ensure(8), "count");
  NDT_CK(launch_count_ge(ctx->snr.as<float>(), ctx->last_n, min_snr, ctx->count_dev.as<unsigned long long>(),
                         ctx->stream), "count kernel");
  ctx->launches += 1;
  unsigned long long c = 0;
  NDT_CK(cudaMemcpyAsync(&c, ctx->count_dev.p, 8, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  *count = (int64_t)c;
  return NDT_OK;
}

ndt_status ndt_predict_positions(ndt_ctx* ctx, const double* states, double t0, int64_t n_orbits,
                                 double* xy_out) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (ctx->n_exp < 1) return fail(ctx, NDT_ESTATE, "predict_positions before load_exposures");
  if (n_orbits < 0 || (n_orbits > 0 && (!states || !xy_out)))
    return fail(ctx, NDT_EINVAL, "bad arguments");
  if (n_orbits == 0) return NDT_OK;
  const void* st_dev = nullptr;
  ndt_status s = to_device(ctx, states, sizeof(double) * 6 * n_orbits, ctx->stage_states, &st_dev);
  if (s != NDT_OK) return s;
  const size_t bytes = sizeof(double) * 2 * (size_t)n_orbits * ctx->n_exp;
  const bool host_out = !is_device_ptr(xy_out);
  double* dst = xy_out;
  if (host_out) {
    NDT_CK(ctx->xy_tmp.ensure(bytes), "position scratch");
    dst = ctx->xy_tmp.as<double>();
  }
  NDT_CK(cudaMemsetAsync(ctx->counters.as<unsigned long long>() + 1, 0, 8, ctx->stream), "memset");
  NDT_CK(launch_predict(static_cast<const double*>(st_dev), n_orbits, t0, ctx->t_ref, ctx->ex_dev.as<ExpDev>(),
                        ctx->pos_to_table_dev.as<int32_t>(), ctx->n_exp, ctx->ph, ctx->state_df != 0, dst,
                        ctx->counters.as<unsigned long long>(), ctx->stream), "predict kernel");
  ctx->launches += 1;
  if (host_out) NDT_CK(cudaMemcpyAsync(xy_out, dst, bytes, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  unsigned long long cnt[2];
  NDT_CK(cudaMemcpy(cnt, ctx->counters.p, 16, cudaMemcpyDeviceToHost), "counters");
  if (cnt[1]) return fail(ctx, NDT_ENOCONV, "%llu Kepler solves did not converge", cnt[1]);
  return NDT_OK;
}

ndt_status ndt_get_planes(ndt_ctx* ctx, int32_t j, float* psi_out, float* phi_out) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (ctx->n_exp < 1) return fail(ctx, NDT_ESTATE, "no exposures loaded");
  if (j < 0 || j >= ctx->n_exp) return fail(ctx, NDT_EINVAL, "exposure %d out of range", j);
  const ExpDev& e = ctx->ex_host[ctx->table_to_sorted[j]];
  const size_t bytes = sizeof(float) * (size_t)e.W * e.H;
  const bool hp = psi_out && !is_device_ptr(psi_out), hf = phi_out && !is_device_ptr(phi_out);
  if (hp || hf) NDT_CK(ctx->xy_tmp.ensure(2 * bytes), "decode scratch");
  float* dp = hp ? ctx->xy_tmp.as<float>() : psi_out;
  float* df = hf ? ctx->xy_tmp.as<float>() + (size_t)e.W * e.H : phi_out;
  NDT_CK(launch_plane_decode(ctx->planes.p, ctx->plane_type, &e, dp, df, ctx->stream), "decode kernel");
  ctx->launches += 1;
  if (hp) NDT_CK(cudaMemcpyAsync(psi_out, dp, bytes, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  if (hf) NDT_CK(cudaMemcpyAsync(phi_out, df, bytes, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  return NDT_OK;
}

ndt_status ndt_set_launch(ndt_ctx* ctx, int32_t mode, int32_t orbit_tile, int32_t exp_tile,
                          int32_t use_graph) {
  if (!ctx) return NDT_EINVAL;
  if (mode != NDT_LAUNCH_PLAIN && mode != NDT_LAUNCH_PERSISTENT)
    return fail(ctx, NDT_EINVAL, "bad launch mode %d", mode);
  if (mode == NDT_LAUNCH_PERSISTENT) {
    if (orbit_tile != 32 && orbit_tile != 64 && orbit_tile != 128)
      return fail(ctx, NDT_EINVAL, "orbit_tile %d not in {32, 64, 128}", orbit_tile);
    if (exp_tile != 8 && exp_tile != 16 && exp_tile != 32)
      return fail(ctx, NDT_EINVAL, "exp_tile %d not in {8, 16, 32}", exp_tile);
    ctx->orbit_tile = orbit_tile;
    ctx->exp_tile = exp_tile;
  }
  ctx->mode = mode;
  ctx->use_graph = use_graph ? 1 : 0;
  return NDT_OK;
}

ndt_status ndt_set_filter_broadening(ndt_ctx* ctx, float sigma_px) {
  if (!ctx) return NDT_EINVAL;
  if (!(sigma_px >= 0.0f) || !std::isfinite(sigma_px))
    return fail(ctx, NDT_EINVAL, "filter broadening %g must be finite and >= 0", sigma_px);
  ctx->broaden = sigma_px;
  return NDT_OK;
}

ndt_status ndt_set_offchip_test(ndt_ctx* ctx, int32_t enabled) {
  if (!ctx) return NDT_EINVAL;
  ctx->offchip = enabled ? 1 : 0;
  return NDT_OK;
}

ndt_status ndt_set_fp64_geometry(ndt_ctx* ctx, int32_t enabled) {
  if (!ctx) return NDT_EINVAL;
  ctx->geometry_fp64 = enabled ? 1 : 0;
  return NDT_OK;
}

ndt_status ndt_set_df_state(ndt_ctx* ctx, int32_t enabled) {
  if (!ctx) return NDT_EINVAL;
  ctx->state_df = enabled ? 1 : 0;
  return NDT_OK;
}

ndt_status ndt_set_footprint_sort(ndt_ctx* ctx, int32_t enabled) {
  if (!ctx) return NDT_EINVAL;
  ctx->footprint = enabled ? 1 : 0;
  return NDT_OK;
}

ndt_status ndt_set_block_test(ndt_ctx* ctx, int32_t enabled) {
  if (!ctx) return NDT_EINVAL;
  ctx->block_test = enabled ? 1 : 0;
  return NDT_OK;
}

ndt_status ndt_autotune(ndt_ctx* ctx, const double* states, double t0, int64_t n_orbits,
                        const int64_t* fam_orbit_off, const int64_t* fam_exp_off,
                        const int32_t* fam_exp_idx, int32_t n_fam, float* times_ms) {
  if (!ctx) return NDT_EINVAL;
  const int32_t saved_mode = ctx->mode, saved_graph = ctx->use_graph;
  const int ots[3] = {32, 64, 128}, ets[3] = {8, 16, 32};
  float best = 1e30f;
  int best_ot = 64, best_et = 16;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      ctx->mode = NDT_LAUNCH_PERSISTENT;
      ctx->orbit_tile = ots[i];
      ctx->exp_tile = ets[j];
      ctx->use_graph = 0;
      float ms_best = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {   // first run warms up
        ndt_status s = ndt_stack_orbits(ctx, states, t0, n_orbits, fam_orbit_off, fam_exp_off,
                                        fam_exp_idx, n_fam, 1, nullptr, nullptr, nullptr, nullptr);
        if (s != NDT_OK) { ctx->mode = saved_mode; ctx->use_graph = saved_graph; return s; }
        NDT_CK(cudaEventSynchronize(ctx->ev[3]), "sync");
        float ms = 0.0f;
        NDT_CK(cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]), "timing");
        if (rep > 0) ms_best = std::min(ms_best, ms);
      }
      if (times_ms) times_ms[3 * i + j] = ms_best;
      if (ms_best < best) { best = ms_best; best_ot = ots[i]; best_et = ets[j]; }
    }
  ctx->mode = saved_mode;
  ctx->use_graph = saved_graph;
  ctx->orbit_tile = best_ot;
  ctx->exp_tile = best_et;
  return NDT_OK;
}

}  // extern "C"

// ------------------------------------------------------------ vetting ----

namespace {

// Output buffer on the device: `user` itself when it is device memory, else a
// context scratch that is copied back by copy_out().
template <class T>
ndt_status out_buffer(ndt_ctx* ctx, T* user, size_t count, DevBuf& scratch, T** dev) {
  if (!user || is_device_ptr(user)) {
    *dev = user;
    return NDT_OK;
  }
  NDT_CK(scratch.ensure(sizeof(T) * count), "output scratch");
  *dev = static_cast<T*>(scratch.p);
  return NDT_OK;
}

template <class T>
ndt_status copy_out(ndt_ctx* ctx, T* user, const T* dev, size_t count) {
  if (user && user != dev)
    NDT_CK(cudaMemcpyAsync(user, dev, sizeof(T) * count, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  return NDT_OK;
}

// Timeout flag of the tensor-core forward (an int after the two counters).
int* cnn_err(ndt_ctx* ctx) { return reinterpret_cast<int*>(ctx->counters.as<unsigned long long>() + 2); }

ndt_status check_cnn_err(ndt_ctx* ctx) {
  int e = 0;
  NDT_CK(cudaMemcpy(&e, cnn_err(ctx), sizeof e, cudaMemcpyDeviceToHost), "flag read");
  if (e) {
    NDT_CK(cudaMemset(cnn_err(ctx), 0, sizeof e), "flag reset");
    return fail(ctx, NDT_ETIMEOUT, "tensor-core CNN forward: a bounded wait timed out");
  }
  return NDT_OK;
}

ndt_status make_stamps(ndt_ctx* ctx, const double* states, double t0, int64_t n_orbits,
                       const int64_t* cand_idx, int64_t n_cand, float* f32_dev,
                       __nv_bfloat16* bf16_dev) {
  if (ctx->n_exp < 1) return fail(ctx, NDT_ESTATE, "stamps before load_exposures");
  if (n_orbits < 0 || n_cand < 0 || (n_cand > 0 && (!states || !cand_idx)))
    return fail(ctx, NDT_EINVAL, "bad stamp arguments");
  if (n_cand == 0) return NDT_OK;
  const void* st_dev = nullptr;
  ndt_status s = to_device(ctx, states, sizeof(double) * 6 * n_orbits, ctx->stage_states, &st_dev);
  if (s != NDT_OK) return s;
  const void* cd = nullptr;
  s = to_device(ctx, cand_idx, sizeof(int64_t) * n_cand, ctx->cand_stage, &cd);
  if (s != NDT_OK) return s;
  NDT_CK(ctx->stamp_pos.ensure(sizeof(int2) * n_cand * ctx->n_exp + sizeof(int) * n_cand), "stamp positions");
  int* pos_cnt = reinterpret_cast<int*>(ctx->stamp_pos.as<int2>() + n_cand * ctx->n_exp);
  // reset the failure counter only: the valid-sample count of the last stack stays
  NDT_CK(cudaMemsetAsync(ctx->counters.as<unsigned long long>() + 1, 0, 8, ctx->stream), "memset");
  NDT_CK(launch_stamp_positions(static_cast<const double*>(st_dev), n_orbits, t0, ctx->t_ref, ctx->state_df != 0,
                                static_cast<const int64_t*>(cd), n_cand, ctx->ex_dev.as<ExpDev>(),
                                ctx->n_exp, ctx->ph, ctx->stamp_pos.as<int2>(), pos_cnt,
                                ctx->counters.as<unsigned long long>(), ctx->stream), "stamp positions");
  NDT_CK(launch_stamps(ctx->stamp_pos.as<int2>(), pos_cnt, n_cand, ctx->ex_dev.as<ExpDev>(), ctx->n_exp,
                       ctx->planes.p, ctx->plane_type, f32_dev, bf16_dev, ctx->n_sms, ctx->stream),
         "stamp kernel");
  ctx->launches += 2;
  return NDT_OK;
}

}  // namespace

extern "C" {

ndt_status ndt_dedup_candidates(ndt_ctx* ctx, const double* states, double t0, int64_t n_orbits,
                                const int64_t* cand_idx, int64_t n_cand, float radius_px, int32_t n_ref,
                                double t_lo, double t_hi, int64_t* keep_idx, int64_t* n_keep) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (ctx->n_exp < 1) return fail(ctx, NDT_ESTATE, "dedup before load_exposures");
  if (!n_keep) return fail(ctx, NDT_EINVAL, "n_keep is null");
  if (n_orbits < 0 || n_cand < 0 || n_cand > (int64_t(1) << 26) ||
      (n_cand > 0 && (!states || !cand_idx || !keep_idx)))
    return fail(ctx, NDT_EINVAL, "bad dedup arguments");
  if (!(radius_px > 0.0f) || !std::isfinite(radius_px) || n_ref < 1 || n_ref > 8)
    return fail(ctx, NDT_EINVAL, "radius %g or n_ref %d out of range", radius_px, n_ref);
  *n_keep = 0;
  if (n_cand == 0) return NDT_OK;
  // reference exposures: evenly spread over the epoch-sorted exposures with
  // epochs in [t_lo, t_hi] (every exposure when the window is empty or NaN)
  int32_t lo = 0, hi = ctx->n_exp - 1;
  if (t_lo <= t_hi) {
    while (lo < ctx->n_exp && ctx->ex_host[lo].t < t_lo) ++lo;
    while (hi >= 0 && ctx->ex_host[hi].t > t_hi) --hi;
    if (lo > hi) return fail(ctx, NDT_EINVAL, "no exposure with an epoch in [%g, %g]", t_lo, t_hi);
  }
  const int32_t m = hi - lo + 1;
  std::vector<int32_t> ref;
  for (int k = 0; k < n_ref; ++k) {
    const int32_t pos = lo + (n_ref == 1 ? (m - 1) / 2 : (int32_t)std::lround((double)k * (m - 1) / (n_ref - 1)));
    if (ref.empty() || pos > ref.back()) ref.push_back(pos);
  }
  const int nr = (int)ref.size();
  const void* st_dev = nullptr;
  ndt_status s = to_device(ctx, states, sizeof(double) * 6 * n_orbits, ctx->stage_states, &st_dev);
  if (s != NDT_OK) return s;
  const void* cd = nullptr;
  if ((s = to_device(ctx, cand_idx, sizeof(int64_t) * n_cand, ctx->cand_stage, &cd)) != NDT_OK) return s;
  int64_t* out = nullptr;
  if ((s = out_buffer(ctx, keep_idx, n_cand, ctx->dedup_out, &out)) != NDT_OK) return s;
  NDT_CK(ctx->dedup_ref.ensure(sizeof(int32_t) * nr + 16), "dedup references");
  NDT_CK(ctx->dedup_scratch.ensure(dedup_scratch_bytes(n_cand, nr, dedup_table_size(n_cand))),
         "dedup scratch");
  NDT_CK(cudaMemcpyAsync(ctx->dedup_ref.p, ref.data(), sizeof(int32_t) * nr, cudaMemcpyHostToDevice,
                         ctx->stream), "upload");
  int* n_keep_dev = reinterpret_cast<int*>(static_cast<unsigned char*>(ctx->dedup_ref.p) +
                                           ((sizeof(int32_t) * nr + 3) / 4) * 4);
  NDT_CK(cudaMemsetAsync(ctx->counters.as<unsigned long long>() + 1, 0, 8, ctx->stream), "memset");
  NDT_CK(launch_dedup(static_cast<const double*>(st_dev), n_orbits, t0, ctx->t_ref, ctx->state_df != 0,
                         static_cast<const int64_t*>(cd),
                      n_cand, ctx->ex_dev.as<ExpDev>(), ctx->dedup_ref.as<int32_t>(), nr, ctx->ph, radius_px,
                      ctx->dedup_scratch.p, ctx->counters.as<unsigned long long>(), out, n_keep_dev,
                      ctx->stream),
         "dedup kernels");
  ctx->launches += 6;
  int nk = 0;
  NDT_CK(cudaMemcpyAsync(&nk, n_keep_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  if ((s = copy_out(ctx, keep_idx, out, (size_t)nk)) != NDT_OK) return s;
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  *n_keep = nk;
  return NDT_OK;
}

ndt_status ndt_selftest_wait_timeout(ndt_ctx* ctx) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const int64_t np = cnn_param_count();
  NDT_CK(ctx->cnn_params.ensure(sizeof(float) * np), "self-test parameters");
  NDT_CK(ctx->cnn_x.ensure(2 * 2 * 441), "self-test stamp");
  NDT_CK(ctx->cnn_out.ensure(sizeof(float)), "self-test logit");
  NDT_CK(cudaMemsetAsync(ctx->cnn_params.p, 0, sizeof(float) * np, ctx->stream), "memset");
  NDT_CK(cudaMemsetAsync(ctx->cnn_x.p, 0, 2 * 2 * 441, ctx->stream), "memset");
  NDT_CK(cudaMemsetAsync(cnn_err(ctx), 0, sizeof(int), ctx->stream), "memset");
  NDT_CK(launch_cnn_forward_tc(ctx->cnn_params.as<float>(), ctx->cnn_x.as<__nv_bfloat16>(), 1,
                               ctx->cnn_out.as<float>(), cnn_err(ctx), 1, ctx->stream,
                               /*withhold_first_layer=*/1),
         "self-test kernel");
  ctx->launches += 1;
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  return check_cnn_err(ctx);
}

ndt_status ndt_noise_mad(ndt_ctx* ctx, const float* const* images, const int64_t* n_pixels,
                         int32_t n_images, int32_t max_rounds, float* median_out, float* sigma_out,
                         int32_t* rounds_out) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (n_images < 0 || (n_images > 0 && (!images || !n_pixels)) || max_rounds < 1 || max_rounds > 100)
    return fail(ctx, NDT_EINVAL, "noise_mad: bad arguments");
  if (n_images == 0) return NDT_OK;
  std::vector<const float*> dev(n_images);
  std::vector<int64_t> npx(n_pixels, n_pixels + n_images);
  int64_t host_total = 0;
  for (int i = 0; i < n_images; ++i) {
    if (npx[i] < 0 || npx[i] > (int64_t)UINT32_MAX || (npx[i] > 0 && !images[i]))
      return fail(ctx, NDT_EINVAL, "noise_mad: image %d", i);
    if (npx[i] > 0 && !is_device_ptr(images[i])) host_total += npx[i];
  }
  if (host_total) NDT_CK(ctx->mad_stage.ensure(sizeof(float) * host_total), "noise staging");
  int64_t off = 0;
  for (int i = 0; i < n_images; ++i) {
    if (npx[i] == 0 || is_device_ptr(images[i])) {
      dev[i] = images[i];
      continue;
    }
    float* dst = ctx->mad_stage.as<float>() + off;
    NDT_CK(cudaMemcpyAsync(dst, images[i], sizeof(float) * npx[i], cudaMemcpyHostToDevice, ctx->stream), "H2D");
    dev[i] = dst;
    off += npx[i];
  }
  std::vector<MadState> st;
  ndt_status s = mad_estimate(ctx, dev, npx, max_rounds, st);
  if (s != NDT_OK) return s;
  std::vector<float> med(n_images), sig(n_images);
  std::vector<int32_t> rnd(n_images);
  for (int i = 0; i < n_images; ++i) {
    med[i] = st[i].m_last;
    sig[i] = st[i].sigma;
    rnd[i] = st[i].rounds;
    if (npx[i] == 0) med[i] = sig[i] = std::numeric_limits<float>::quiet_NaN();
  }
  auto put = [&](auto* user, const auto& v) -> ndt_status {
    if (!user) return NDT_OK;
    const size_t bytes = sizeof(v[0]) * v.size();
    if (is_device_ptr(user)) {
      NDT_CK(cudaMemcpyAsync(user, v.data(), bytes, cudaMemcpyHostToDevice, ctx->stream), "output H2D");
    } else {
      std::memcpy(user, v.data(), bytes);
    }
    return NDT_OK;
  };
  if ((s = put(median_out, med)) != NDT_OK) return s;
  if ((s = put(sigma_out, sig)) != NDT_OK) return s;
  if ((s = put(rounds_out, rnd)) != NDT_OK) return s;
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  return NDT_OK;
}

ndt_status ndt_trim_candidates(ndt_ctx* ctx, const double* states, double t0, int64_t n_orbits,
                               const int64_t* cand_idx, int64_t n_cand, float kappa, int32_t max_iter,
                               int32_t min_obs, float* nu_out, int32_t* nkept_out) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (ctx->n_exp < 1) return fail(ctx, NDT_ESTATE, "trim_candidates before load_exposures");
  if (!(kappa > 0.0f) || max_iter < 1 || max_iter > 1000 || min_obs < 0)
    return fail(ctx, NDT_EINVAL, "trim: kappa %g, max_iter %d, min_obs %d", kappa, max_iter, min_obs);
  if (n_orbits < 0 || n_cand < 0 || (n_cand > 0 && (!states || !cand_idx || !nu_out)))
    return fail(ctx, NDT_EINVAL, "bad trim arguments");
  if (n_cand == 0) return NDT_OK;
  const void* st_dev = nullptr;
  ndt_status s = to_device(ctx, states, sizeof(double) * 6 * n_orbits, ctx->stage_states, &st_dev);
  if (s != NDT_OK) return s;
  const void* cd = nullptr;
  if ((s = to_device(ctx, cand_idx, sizeof(int64_t) * n_cand, ctx->cand_stage, &cd)) != NDT_OK) return s;
  float* nu = nullptr;
  int32_t* nk = nullptr;
  if ((s = out_buffer(ctx, nu_out, (size_t)n_cand, ctx->trim_nu, &nu)) != NDT_OK) return s;
  if ((s = out_buffer(ctx, nkept_out, (size_t)n_cand, ctx->trim_n, &nk)) != NDT_OK) return s;
  NDT_CK(ctx->stamp_pos.ensure(sizeof(int2) * n_cand * ctx->n_exp + sizeof(int) * n_cand), "trim positions");
  int* pos_cnt = reinterpret_cast<int*>(ctx->stamp_pos.as<int2>() + n_cand * ctx->n_exp);
  NDT_CK(ctx->trim_bits.ensure(4 * trim_scratch_words(n_cand, ctx->n_exp)), "trim scratch");
  NDT_CK(cudaMemsetAsync(ctx->counters.as<unsigned long long>() + 1, 0, 8, ctx->stream), "memset");
  NDT_CK(launch_stamp_positions(static_cast<const double*>(st_dev), n_orbits, t0, ctx->t_ref, ctx->state_df != 0,
                                static_cast<const int64_t*>(cd), n_cand, ctx->ex_dev.as<ExpDev>(),
                                ctx->n_exp, ctx->ph, ctx->stamp_pos.as<int2>(), pos_cnt,
                                ctx->counters.as<unsigned long long>(), ctx->stream), "trim positions");
  NDT_CK(launch_trim(ctx->stamp_pos.as<int2>(), pos_cnt, n_cand, ctx->ex_dev.as<ExpDev>(), ctx->n_exp, ctx->planes.p,
                     ctx->plane_type, kappa, max_iter, min_obs, ctx->trim_bits.as<uint32_t>(), nu, nk, nullptr,
                     nullptr, ctx->n_sms, ctx->stream),
         "trim kernel");
  ctx->launches += 2;
  if ((s = copy_out(ctx, nu_out, nu, (size_t)n_cand)) != NDT_OK) return s;
  if ((s = copy_out(ctx, nkept_out, nk, (size_t)n_cand)) != NDT_OK) return s;
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  return NDT_OK;
}

ndt_status ndt_stamps(ndt_ctx* ctx, const double* states, double t0, int64_t n_orbits,
                      const int64_t* cand_idx, int64_t n_cand, float* stamps_f32,
                      uint16_t* stamps_bf16) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const size_t cnt = (size_t)n_cand * 2 * 441;
  float* f = nullptr;
  uint16_t* b = nullptr;
  ndt_status s = out_buffer(ctx, stamps_f32, cnt, ctx->stamp_f32, &f);
  if (s == NDT_OK) s = out_buffer(ctx, stamps_bf16, cnt, ctx->stamp_bf16, &b);
  if (s == NDT_OK)
    s = make_stamps(ctx, states, t0, n_orbits, cand_idx, n_cand, f,
                    reinterpret_cast<__nv_bfloat16*>(b));
  if (s != NDT_OK) return s;
  if ((s = copy_out(ctx, stamps_f32, f, cnt)) != NDT_OK) return s;
  if ((s = copy_out(ctx, stamps_bf16, b, cnt)) != NDT_OK) return s;
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  return NDT_OK;
}

int64_t ndt_cnn_param_count(void) { return cnn_param_count(); }

ndt_status ndt_cnn_forward(ndt_ctx* ctx, const float* params, const uint16_t* stamps_bf16,
                           int64_t n, float* logits) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (n < 0 || (n > 0 && (!params || !stamps_bf16 || !logits))) return fail(ctx, NDT_EINVAL, "bad CNN arguments");
  if (n == 0) return NDT_OK;
  const void* th = nullptr;
  const void* x = nullptr;
  ndt_status s = to_device(ctx, params, sizeof(float) * cnn_param_count(), ctx->cnn_params, &th);
  if (s == NDT_OK) s = to_device(ctx, stamps_bf16, sizeof(uint16_t) * 2 * 441 * n, ctx->cnn_x, &x);
  float* lo = nullptr;
  if (s == NDT_OK) s = out_buffer(ctx, logits, n, ctx->cnn_out, &lo);
  if (s != NDT_OK) return s;
  NDT_CK(launch_cnn_forward_tc(static_cast<const float*>(th), static_cast<const __nv_bfloat16*>(x), n, lo,
                               cnn_err(ctx), ctx->n_sms, ctx->stream), "CNN forward");
  ctx->launches += 1;
  if ((s = copy_out(ctx, logits, lo, n)) != NDT_OK) return s;
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  return check_cnn_err(ctx);
}

ndt_status ndt_cnn_loss_grad(ndt_ctx* ctx, const float* params, const uint16_t* stamps_bf16,
                             const float* labels, int64_t n, float* grad, float* loss_out,
                             float* logits_out) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (n < 1 || !params || !stamps_bf16 || !labels || !grad)
    return fail(ctx, NDT_EINVAL, "bad CNN arguments");
  const int np = cnn_param_count();
  const void *th = nullptr, *x = nullptr, *lab = nullptr;
  ndt_status s = to_device(ctx, params, sizeof(float) * np, ctx->cnn_params, &th);
  if (s == NDT_OK) s = to_device(ctx, stamps_bf16, sizeof(uint16_t) * 2 * 441 * n, ctx->cnn_x, &x);
  if (s == NDT_OK) s = to_device(ctx, labels, sizeof(float) * n, ctx->cnn_labels, &lab);
  float* g = nullptr;
  if (s == NDT_OK) s = out_buffer(ctx, grad, np, ctx->cnn_grad, &g);
  if (s != NDT_OK) return s;
  // scratch: loss (1 float, padded) + logits (n) + one a1 plane set per CTA
  const int blocks = cnn_backward_blocks(n, ctx->n_sms);
  NDT_CK(ctx->cnn_scratch.ensure(sizeof(float) * (16 + n + (size_t)blocks * 32 * 441)), "CNN scratch");
  float* loss_d = ctx->cnn_scratch.as<float>();
  float* logit_d = loss_d + 16;
  float* a1 = logit_d + n;
  NDT_CK(cudaMemsetAsync(g, 0, sizeof(float) * np, ctx->stream), "memset");
  NDT_CK(cudaMemsetAsync(loss_d, 0, sizeof(float), ctx->stream), "memset");
  NDT_CK(launch_cnn_backward(static_cast<const float*>(th), static_cast<const __nv_bfloat16*>(x),
                             static_cast<const float*>(lab), n, g, loss_d, a1, logit_d, ctx->n_sms,
                             ctx->stream), "CNN backward");
  ctx->launches += 1;
  if ((s = copy_out(ctx, grad, g, np)) != NDT_OK) return s;
  if (loss_out) {
    if (is_device_ptr(loss_out))
      NDT_CK(cudaMemcpyAsync(loss_out, loss_d, 4, cudaMemcpyDeviceToDevice, ctx->stream), "copy");
    else
      NDT_CK(cudaMemcpyAsync(loss_out, loss_d, 4, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  }
  if (logits_out)
    NDT_CK(cudaMemcpyAsync(logits_out, logit_d, sizeof(float) * n,
                           is_device_ptr(logits_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           ctx->stream), "copy");
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  return NDT_OK;
}

ndt_status ndt_cnn_adam_step(ndt_ctx* ctx, float* params, const float* grad, float* m, float* v,
                             int64_t n_params, int32_t step, float lr, float beta1, float beta2,
                             float eps) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (n_params < 1 || n_params > (1 << 30) || step < 1 || !(lr > 0.0f))
    return fail(ctx, NDT_EINVAL, "bad Adam arguments");
  if (!is_device_ptr(params) || !is_device_ptr(grad) || !is_device_ptr(m) || !is_device_ptr(v))
    return fail(ctx, NDT_EINVAL, "Adam state must be device memory");
  NDT_CK(launch_adam(params, grad, m, v, (int)n_params, lr, beta1, beta2, eps, step, ctx->stream),
         "Adam kernel");
  ctx->launches += 1;
  return NDT_OK;
}

ndt_status ndt_vet(ndt_ctx* ctx, const float* params, const double* states, double t0,
                   int64_t n_orbits, const int64_t* cand_idx, int64_t n_cand, float* scores) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (n_cand < 0 || (n_cand > 0 && (!params || !scores))) return fail(ctx, NDT_EINVAL, "bad vet arguments");
  if (n_cand == 0) return NDT_OK;
  NDT_CK(ctx->stamp_bf16.ensure(sizeof(uint16_t) * 2 * 441 * n_cand), "stamp buffer");
  ndt_status s = make_stamps(ctx, states, t0, n_orbits, cand_idx, n_cand, nullptr,
                             ctx->stamp_bf16.as<__nv_bfloat16>());
  if (s != NDT_OK) return s;
  const void* th = nullptr;
  s = to_device(ctx, params, sizeof(float) * cnn_param_count(), ctx->cnn_params, &th);
  float* lo = nullptr;
  if (s == NDT_OK) s = out_buffer(ctx, scores, n_cand, ctx->cnn_out, &lo);
  if (s != NDT_OK) return s;
  NDT_CK(launch_cnn_forward_tc(static_cast<const float*>(th), ctx->stamp_bf16.as<__nv_bfloat16>(), n_cand,
                               lo, cnn_err(ctx), ctx->n_sms, ctx->stream), "CNN forward");
  NDT_CK(launch_sigmoid(lo, n_cand, ctx->stream), "sigmoid");
  ctx->launches += 2;
  if ((s = copy_out(ctx, scores, lo, n_cand)) != NDT_OK) return s;
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  return check_cnn_err(ctx);
}

ndt_status ndt_get_stats(ndt_ctx* ctx, ndt_stats* out) {
  if (!ctx || !out) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  std::memset(out, 0, sizeof *out);
  unsigned long long cnt[5];
  NDT_CK(cudaMemcpy(cnt, ctx->counters.p, 40, cudaMemcpyDeviceToHost), "counters");
  out->kernel_launches = ctx->launches;
  out->offchip_skipped = (int64_t)cnt[3];
  out->block_skipped = (int64_t)cnt[4];
  out->noise_bytes_read = ctx->noise_bytes_read;
  out->samples = ctx->samples;
  out->valid_samples = (int64_t)cnt[0];
  out->kepler_failures = (int64_t)cnt[1];
  if (ctx->have_stack_ev) cudaEventElapsedTime(&out->last_stack_ms, ctx->ev[2], ctx->ev[3]);
  if (ctx->have_planes_ev) cudaEventElapsedTime(&out->last_planes_ms, ctx->ev[0], ctx->ev[1]);
  if (ctx->have_topk_ev) cudaEventElapsedTime(&out->last_topk_ms, ctx->ev[4], ctx->ev[5]);
  out->orbit_tile = ctx->orbit_tile;
  out->exp_tile = ctx->exp_tile;
  out->launch_mode = ctx->mode;
  out->plane_dtype = ctx->plane_type;
  return NDT_OK;
}

ndt_status ndt_synchronize(ndt_ctx* ctx) {
  if (!ctx) return NDT_EINVAL;
  NDT_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  NDT_CK(cudaStreamSynchronize(ctx->stream), "sync");
  return NDT_OK;
}

}  // extern "C"
