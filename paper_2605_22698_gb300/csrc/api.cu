// C ABI of the library: errors, workspaces, model handles, the neighbour
// entry point and the energy/forces entry point (plain FP32 form here; the
// fused BF16 form lives in fused_bf16.cu).
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <fstream>

#include "launchers.cuh"
#include "profile.cuh"

namespace mlip {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
const char* last_error() { return g_err; }

int Workspace::get(const std::string& name, size_t bytes, void** out) {
  Buf& b = bufs[name];
  if (b.bytes < bytes) {
    // stream-ordered: the old buffer is released once the work queued before
    // on this workspace's stream has finished (no device-wide synchronisation,
    // which would fail while another thread captures a CUDA graph)
    if (b.p) {
      cudaError_t e = cudaFreeAsync(b.p, stream);
      if (e != cudaSuccess) { set_error("workspace release: %s", cudaGetErrorString(e)); return MLIP_ERR_CUDA; }
      b.p = nullptr;
      b.bytes = 0;
    }
    size_t nb = bytes + bytes / 8;
    ++gen;
    cudaError_t e = cudaMallocAsync(&b.p, nb, stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("workspace '%s': cudaMalloc of %zu bytes failed: %s", name.c_str(), nb, cudaGetErrorString(e));
      b.p = nullptr;
      return MLIP_ERR_OOM;
    }
    b.bytes = nb;
  }
  *out = b.p;
  return MLIP_OK;
}

void Workspace::release() {
  cudaStreamSynchronize(stream);
  for (auto& kv : bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  bufs.clear();
}

int HostStage::get(size_t need, void** out) {
  if (bytes < need) {
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMallocHost(&p, need);
    if (e != cudaSuccess) { cudaGetLastError(); set_error("pinned staging: %s", cudaGetErrorString(e)); return MLIP_ERR_OOM; }
    bytes = need;
  }
  *out = p;
  return MLIP_OK;
}
HostStage::~HostStage() {
  if (p) cudaFreeHost(p);
}

static int count_paths(int L, int Lsh, int* P0, bool all_parities = false) {
  int P = 0, p0 = 0;
  for (int l1 = 0; l1 <= L; ++l1)
    for (int l2 = 0; l2 <= Lsh; ++l2)
      for (int l3 = 0; l3 <= L; ++l3)
        if (l3 >= std::abs(l1 - l2) && l3 <= l1 + l2 && (all_parities || (l1 + l2 + l3) % 2 == 0)) {
          ++P;
          if (l1 == 0) ++p0;
        }
  if (P0) *P0 = p0;
  return P;
}

static int64_t weights_for(const mlip_model_desc& d, int P) {
  const int64_t S = d.n_species, C = d.channels, H = d.hidden, NB = d.n_basis, L = d.l_max;
  const int64_t sc = d.correlation == 2 ? S * (L + 1 + sc_num_paths(d.l_max)) * C : 0;
  const int64_t gt = d.gate ? S * (L + 1) * C * C + C * L * C + S * C * L * C : 0;
  return S * C + d.n_layers * (NB * H + H * H + H * P * C + (L + 1) * C * C + sc + gt) + S * C + S +
         (d.charges ? S * C + S : 0);
}

static int validate_desc(const mlip_model_desc* d, int precision) {
  if (!d) { set_error("null model description"); return MLIP_ERR_INVALID_ARG; }
  if (d->n_species < 1 || d->n_species > 128) { set_error("n_species %d out of range", d->n_species); return MLIP_ERR_INVALID_ARG; }
  if (d->n_layers < 1 || d->n_layers > 8) { set_error("n_layers %d out of range", d->n_layers); return MLIP_ERR_INVALID_ARG; }
  if (d->channels != 16 && d->channels != 32 && d->channels != 64 && d->channels != 128) {
    set_error("channels %d unsupported (16, 32, 64, 128)", d->channels);
    return MLIP_ERR_INVALID_ARG;
  }
  if (d->l_max != 2 && d->l_max != 3) { set_error("l_max %d unsupported (2, 3)", d->l_max); return MLIP_ERR_INVALID_ARG; }
  if (d->sh_l_max != 3) { set_error("sh_l_max must be 3"); return MLIP_ERR_INVALID_ARG; }
  if (d->n_basis != 8) { set_error("n_basis must be 8"); return MLIP_ERR_INVALID_ARG; }
  if (d->hidden != 32 && d->hidden != 64) { set_error("hidden %d unsupported (32, 64)", d->hidden); return MLIP_ERR_INVALID_ARG; }
  if (d->envelope_p < 1 || d->envelope_p > 16) { set_error("envelope_p %d out of range", d->envelope_p); return MLIP_ERR_INVALID_ARG; }
  if (d->correlation != 0 && d->correlation != 2) {
    set_error("correlation %d unsupported (0: none, 2: symmetric contraction of order 2)", d->correlation);
    return MLIP_ERR_INVALID_ARG;
  }
  if (d->charges != 0 && d->charges != 1) { set_error("charges must be 0 or 1"); return MLIP_ERR_INVALID_ARG; }
  if (d->gate != 0 && d->gate != 1) { set_error("gate must be 0 or 1"); return MLIP_ERR_INVALID_ARG; }
  if (d->gate && d->channels < 32) { set_error("the gated update needs 32, 64 or 128 channels"); return MLIP_ERR_INVALID_ARG; }
  if (d->parity != 0 && d->parity != 1) { set_error("parity must be 0 or 1"); return MLIP_ERR_INVALID_ARG; }
  if (d->parity && (d->correlation || d->charges || d->gate)) {
    set_error("mixed parity (parity = 1) is built without the contraction, the charge head and the gate");
    return MLIP_ERR_INVALID_ARG;
  }
  if (d->parity && precision != MLIP_PREC_FP32) {
    set_error("mixed parity (parity = 1) runs in the plain FP32 form");
    return MLIP_ERR_INVALID_ARG;
  }
  if (d->charges && !(d->coulomb_r0 > 0.0 && d->coulomb_r0 < 1e3)) {
    set_error("coulomb_r0 %g out of range (0, 1000)", d->coulomb_r0);
    return MLIP_ERR_INVALID_ARG;
  }
  if (!(d->cutoff > 0) || !(d->avg_num_neighbors > 0)) { set_error("cutoff and avg_num_neighbors must be positive"); return MLIP_ERR_INVALID_ARG; }
  if (precision != MLIP_PREC_FP32 && precision != MLIP_PREC_BF16 && precision != MLIP_PREC_F16) {
    set_error("unknown precision %d", precision);
    return MLIP_ERR_INVALID_ARG;
  }
  if (precision != MLIP_PREC_FP32 && (d->channels != 128 || d->hidden != 64)) {
    set_error("the fused tensor-core form needs 128 channels and hidden width 64");
    return MLIP_ERR_INVALID_ARG;
  }
  return MLIP_OK;
}

}  // namespace mlip

using namespace mlip;

extern "C" {

const char* mlip_last_error(void) { return last_error(); }
int mlip_version(void) { return 1; }

int mlip_model_num_weights(const mlip_model_desc* desc, int64_t* n_weights) {
  MLIP_TRY(validate_desc(desc, MLIP_PREC_FP32));
  *n_weights = weights_for(*desc, count_paths(desc->l_max, desc->sh_l_max, nullptr));
  return MLIP_OK;
}

int mlip_model_create(const mlip_model_desc* desc, const float* weights, int64_t n_weights, int precision,
                      mlip_model** out) {
  if (!out || !weights) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  *out = nullptr;
  MLIP_TRY(validate_desc(desc, precision));
  int P0 = 0;
  const int P = count_paths(desc->l_max, desc->sh_l_max, &P0, desc->parity != 0);
  const int64_t need = weights_for(*desc, P);
  if (n_weights != need) { set_error("expected %lld weights, got %lld", (long long)need, (long long)n_weights); return MLIP_ERR_INVALID_ARG; }
  mlip_model* M = new mlip_model();
  M->S = desc->n_species; M->T = desc->n_layers; M->C = desc->channels; M->L = desc->l_max;
  M->Lsh = desc->sh_l_max; M->NB = desc->n_basis; M->H = desc->hidden; M->p = desc->envelope_p;
  M->rc = desc->cutoff; M->avg_nb = desc->avg_num_neighbors;
  M->P = P; M->P0 = P0; M->D = (M->L + 1) * (M->L + 1);
  M->corr = desc->correlation;
  M->charges = desc->charges;
  M->gate = desc->gate;
  M->parity = desc->parity;
  M->r0 = desc->coulomb_r0;
  M->Q = M->corr == 2 ? sc_num_paths(M->L) : 0;
  M->precision = precision;
  if (desc->masses) M->masses.assign(desc->masses, desc->masses + M->S);
  M->host_weights.assign(weights, weights + n_weights);
  if (M->parity) {
    // the mixed-parity model's definition: embedding and readout on the even
    // scalars only, block-diagonal channel mixes; the other weights are zeroed
    float* w = M->host_weights.data();
    const int64_t S = M->S, C = M->C, H = M->H, NB = M->NB, Ch = C / 2;
    int64_t off = 0;
    for (int64_t z = 0; z < S; ++z)
      for (int64_t c = Ch; c < C; ++c) w[z * C + c] = 0.0f;
    off += S * C;
    for (int t = 0; t < M->T; ++t) {
      off += NB * H + H * H + H * (int64_t)P * C;
      for (int l = 0; l <= M->L; ++l)
        for (int64_t c1 = 0; c1 < C; ++c1)
          for (int64_t c2 = 0; c2 < C; ++c2)
            if ((c1 < Ch) != (c2 < Ch)) w[off + ((int64_t)l * C + c1) * C + c2] = 0.0f;
      off += (int64_t)(M->L + 1) * C * C;
    }
    for (int64_t z = 0; z < S; ++z)
      for (int64_t c = Ch; c < C; ++c) w[off + z * C + c] = 0.0f;
    weights = w;
  }
  cudaGetDevice(&M->device);
  cudaError_t e = cudaMalloc(&M->d_weights, sizeof(float) * n_weights);
  if (e != cudaSuccess) { cudaGetLastError(); delete M; set_error("cudaMalloc weights: %s", cudaGetErrorString(e)); return MLIP_ERR_OOM; }
  e = cudaMemcpy(M->d_weights, weights, sizeof(float) * n_weights, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cudaFree(M->d_weights); delete M; set_error("copy weights: %s", cudaGetErrorString(e)); return MLIP_ERR_CUDA; }
  const float* q = M->d_weights;
  const int64_t S = M->S, C = M->C, H = M->H, NB = M->NB;
  M->W_emb = q; q += S * C;
  for (int t = 0; t < M->T; ++t) {
    M->W1.push_back(q); q += NB * H;
    M->W2.push_back(q); q += H * H;
    M->W3.push_back(q); q += H * P * C;
    M->Wmix.push_back(q); q += (int64_t)(M->L + 1) * C * C;
    if (M->corr == 2) {
      M->Wsc1.push_back(q); q += S * (M->L + 1) * C;
      M->Wsc2.push_back(q); q += S * M->Q * C;
    }
    if (M->gate) {
      const int64_t LC = (int64_t)M->L * C;
      M->Wself.push_back(q); q += S * (M->L + 1) * C * C;
      M->Wgate.push_back(q); q += C * LC;
      M->Wselfgate.push_back(q); q += S * C * LC;
    }
  }
  M->W_out = q; q += S * C;
  M->E0 = q; q += S;
  if (M->charges) {
    M->W_q = q; q += S * C;
    M->q0 = q; q += S;
  }
  {  // W_l^T of every layer and order, for the adjoint of the mixes
    const size_t per = (size_t)(M->L + 1) * C * C;
    std::vector<float> wt(per * M->T);
    for (int t = 0; t < M->T; ++t) {
      const float* w = M->host_weights.data() + (M->Wmix[t] - M->d_weights);
      for (int l = 0; l <= M->L; ++l)
        for (int64_t a = 0; a < C; ++a)
          for (int64_t b = 0; b < C; ++b) wt[t * per + l * C * C + b * C + a] = w[l * C * C + a * C + b];
    }
    e = cudaMalloc(&M->d_wmixT, sizeof(float) * wt.size());
    if (e == cudaSuccess) e = cudaMemcpy(M->d_wmixT, wt.data(), sizeof(float) * wt.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("transposed mix weights: %s", cudaGetErrorString(e));
      mlip_model_free(M);
      return MLIP_ERR_OOM;
    }
    for (int t = 0; t < M->T; ++t) M->WmixT.push_back(M->d_wmixT + t * per);
  }
  if (M->gate) {  // transposed gate and self-connection weights for the adjoint; kernel limits
    const int64_t LC = (int64_t)M->L * C, L1 = M->L + 1;
    const size_t per = (size_t)(S * L1 * C * C + LC * C + S * LC * C);
    std::vector<float> wt(per * M->T);
    for (int t = 0; t < M->T; ++t) {
      float* o = wt.data() + t * per;
      const float* ws = M->host_weights.data() + (M->Wself[t] - M->d_weights);
      const float* wg = M->host_weights.data() + (M->Wgate[t] - M->d_weights);
      const float* wsg = M->host_weights.data() + (M->Wselfgate[t] - M->d_weights);
      for (int64_t zl = 0; zl < S * L1; ++zl)
        for (int64_t a = 0; a < C; ++a)
          for (int64_t b = 0; b < C; ++b) o[zl * C * C + b * C + a] = ws[zl * C * C + a * C + b];
      o += S * L1 * C * C;
      for (int64_t a = 0; a < C; ++a)
        for (int64_t b = 0; b < LC; ++b) o[b * C + a] = wg[a * LC + b];
      o += LC * C;
      for (int64_t z = 0; z < S; ++z)
        for (int64_t a = 0; a < C; ++a)
          for (int64_t b = 0; b < LC; ++b) o[z * LC * C + b * C + a] = wsg[z * C * LC + a * LC + b];
    }
    e = cudaMalloc(&M->d_gateT, sizeof(float) * wt.size());
    if (e == cudaSuccess) e = cudaMemcpy(M->d_gateT, wt.data(), sizeof(float) * wt.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("transposed gate weights: %s", cudaGetErrorString(e));
      mlip_model_free(M);
      return MLIP_ERR_OOM;
    }
    for (int t = 0; t < M->T; ++t) {
      const float* base = M->d_gateT + t * per;
      M->WselfT.push_back(base);
      M->WgateT.push_back(base + S * L1 * C * C);
      M->WselfgateT.push_back(base + S * L1 * C * C + LC * C);
    }
    const int rc = gate_prepare(M->L, C);
    if (rc != MLIP_OK) { mlip_model_free(M); return rc; }
  }
  if (precision != MLIP_PREC_FP32) {
    std::vector<uint8_t> all, img;
    for (int t = 0; t < M->T; ++t) {
      std::vector<size_t> goff;
      pack_w3_groups(M, t, img, goff);
      M->w3_layer_off.push_back(all.size());
      M->w3_goff.push_back(goff);
      all.insert(all.end(), img.begin(), img.end());
    }
    {  // split FP16 images of the mix weights
      std::vector<uint8_t> imgs, f, b;
      std::vector<float> scales, sc;
      const size_t per = (size_t)(M->L + 1) * 2 * 128 * 128 * 2;
      for (int t = 0; t < M->T; ++t) {
        pack_mix_images(M->host_weights.data() + (M->Wmix[t] - M->d_weights), M->L, f, b, sc);
        imgs.insert(imgs.end(), f.begin(), f.end());
        imgs.insert(imgs.end(), b.begin(), b.end());
        scales.insert(scales.end(), sc.begin(), sc.end());
      }
      cudaError_t e2 = cudaMalloc(&M->d_miximg, imgs.size());
      if (e2 == cudaSuccess) e2 = cudaMemcpy(M->d_miximg, imgs.data(), imgs.size(), cudaMemcpyHostToDevice);
      if (e2 == cudaSuccess) e2 = cudaMalloc(&M->d_mixscale, sizeof(float) * scales.size());
      if (e2 == cudaSuccess)
        e2 = cudaMemcpy(M->d_mixscale, scales.data(), sizeof(float) * scales.size(), cudaMemcpyHostToDevice);
      if (e2 != cudaSuccess) {
        cudaGetLastError();
        set_error("tensor-core mix weight images: %s", cudaGetErrorString(e2));
        mlip_model_free(M);
        return MLIP_ERR_OOM;
      }
      for (int t = 0; t < M->T; ++t) {
        M->mix_fwd_img.push_back(M->d_miximg + (2 * t) * per);
        M->mix_bwd_img.push_back(M->d_miximg + (2 * t + 1) * per);
        M->mix_scale.push_back(M->d_mixscale + (size_t)t * (M->L + 1));
      }
    }
    if (M->gate) {  // split FP16 weight blocks of the tensor-core gate, per layer: forward, then adjoint
      std::vector<uint8_t> imgs, f, b;
      std::vector<float> scales, sf, sb;
      std::vector<size_t> off;
      for (int t = 0; t < M->T; ++t) {
        const float* hw = M->host_weights.data();
        const float *wm = hw + (M->Wmix[t] - M->d_weights), *wsf = hw + (M->Wself[t] - M->d_weights),
                    *wg = hw + (M->Wgate[t] - M->d_weights), *wsg = hw + (M->Wselfgate[t] - M->d_weights);
        pack_gate_images(false, wm, wsf, wg, wsg, M->L, M->S, f, sf);
        pack_gate_images(true, wm, wsf, wg, wsg, M->L, M->S, b, sb);
        off.push_back(imgs.size());
        imgs.insert(imgs.end(), f.begin(), f.end());
        off.push_back(imgs.size());
        imgs.insert(imgs.end(), b.begin(), b.end());
        scales.insert(scales.end(), sf.begin(), sf.end());
        scales.insert(scales.end(), sb.begin(), sb.end());
      }
      cudaError_t e2 = cudaMalloc(&M->d_gateimg, imgs.size());
      if (e2 == cudaSuccess) e2 = cudaMemcpy(M->d_gateimg, imgs.data(), imgs.size(), cudaMemcpyHostToDevice);
      if (e2 == cudaSuccess) e2 = cudaMalloc(&M->d_gatescale, sizeof(float) * scales.size());
      if (e2 == cudaSuccess)
        e2 = cudaMemcpy(M->d_gatescale, scales.data(), sizeof(float) * scales.size(), cudaMemcpyHostToDevice);
      if (e2 != cudaSuccess) {
        cudaGetLastError();
        set_error("tensor-core gate weight images: %s", cudaGetErrorString(e2));
        mlip_model_free(M);
        return MLIP_ERR_OOM;
      }
      const size_t per = (size_t)(M->L + 1) * 4;
      for (int t = 0; t < M->T; ++t) {
        M->gate_fwd_img.push_back(M->d_gateimg + off[2 * t]);
        M->gate_bwd_img.push_back(M->d_gateimg + off[2 * t + 1]);
        M->gate_fwd_scale.push_back(M->d_gatescale + (2 * t) * per);
        M->gate_bwd_scale.push_back(M->d_gatescale + (2 * t + 1) * per);
      }
      const int rc = gate_tc_prepare();
      if (rc != MLIP_OK) { mlip_model_free(M); return rc; }
    }
    {  // per-species max |W_emb row|
      std::vector<float> em(M->S, 0.0f);
      const float* We = M->host_weights.data() + (M->W_emb - M->d_weights);
      for (int z = 0; z < M->S; ++z)
        for (int c = 0; c < M->C; ++c) em[z] = std::max(em[z], std::fabs(We[(size_t)z * M->C + c]));
      cudaError_t e2 = cudaMalloc(&M->d_embmax, sizeof(float) * std::max(M->S, 1));
      if (e2 == cudaSuccess) e2 = cudaMemcpy(M->d_embmax, em.data(), sizeof(float) * M->S, cudaMemcpyHostToDevice);
      if (e2 != cudaSuccess) {
        cudaGetLastError();
        set_error("embedding maxima: %s", cudaGetErrorString(e2));
        mlip_model_free(M);
        return MLIP_ERR_OOM;
      }
    }
    if (M->H == 64) {  // split FP16 images of the radial MLP's hidden layer (the fused form needs H = 64)
      std::vector<uint8_t> imgs, img1;
      for (int t = 0; t < M->T; ++t) {
        float sc = 1.0f;
        pack_radial_images(M->host_weights.data() + (M->W2[t] - M->d_weights), img1, &sc);
        imgs.insert(imgs.end(), img1.begin(), img1.end());
        M->rad_scale.push_back(sc);
      }
      cudaError_t e2 = cudaMalloc(&M->d_radimg, imgs.size());
      if (e2 == cudaSuccess) e2 = cudaMemcpy(M->d_radimg, imgs.data(), imgs.size(), cudaMemcpyHostToDevice);
      if (e2 != cudaSuccess) {
        cudaGetLastError();
        set_error("tensor-core radial weight images: %s", cudaGetErrorString(e2));
        mlip_model_free(M);
        return MLIP_ERR_OOM;
      }
    }
    e = cudaMalloc(&M->d_w3img, all.size());
    if (e == cudaSuccess) e = cudaMemcpy(M->d_w3img, all.data(), all.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("tensor-core weight image: %s", cudaGetErrorString(e));
      mlip_model_free(M);
      return MLIP_ERR_OOM;
    }
  }
  *out = M;
  return MLIP_OK;
}

int mlip_selftest(int which, double* result) {
  if (!result) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  if (which == 1) return umma_selftest_run(result);
  if (which == 2 || which == 3) return umma_selftest_mn_run(which - 2, result);
  set_error("unknown self test %d", which);
  return MLIP_ERR_INVALID_ARG;
}

int mlip_model_load(const char* path, int precision, mlip_model** out) {
  if (!path || !out) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  std::ifstream f(path, std::ios::binary);
  if (!f) { set_error("cannot open '%s'", path); return MLIP_ERR_NOT_FOUND; }
  char magic[8];
  uint32_t version = 0;
  int32_t hyper[8], corr = 0, charges = 0, gate = 0, parity = 0;
  double dh[2], r0 = 0.0;
  f.read(magic, 8);
  f.read(reinterpret_cast<char*>(&version), 4);
  f.read(reinterpret_cast<char*>(hyper), sizeof(hyper));
  if (version >= 2) {
    f.read(reinterpret_cast<char*>(&corr), 4);
    f.read(reinterpret_cast<char*>(&charges), 4);
    f.read(reinterpret_cast<char*>(&r0), 8);
    f.read(reinterpret_cast<char*>(&gate), 4);
  }
  if (version >= 3) f.read(reinterpret_cast<char*>(&parity), 4);
  f.read(reinterpret_cast<char*>(dh), sizeof(dh));
  if (!f || std::memcmp(magic, "MLIPPRM1", 8) != 0 || version < 1 || version > 3) { set_error("'%s' is not a parameter file", path); return MLIP_ERR_INVALID_ARG; }
  if (hyper[0] < 1 || hyper[0] > 128) { set_error("bad species count"); return MLIP_ERR_INVALID_ARG; }
  std::vector<double> masses(hyper[0]);
  f.read(reinterpret_cast<char*>(masses.data()), sizeof(double) * masses.size());
  int64_t count = 0;
  f.read(reinterpret_cast<char*>(&count), 8);
  if (!f || count < 0 || count > (int64_t)1 << 32) { set_error("truncated parameter file"); return MLIP_ERR_INVALID_ARG; }
  std::vector<float> w(count);
  f.read(reinterpret_cast<char*>(w.data()), sizeof(float) * count);
  if (!f) { set_error("truncated parameter file"); return MLIP_ERR_INVALID_ARG; }
  mlip_model_desc d{hyper[0], hyper[1], hyper[2], hyper[3], hyper[4], hyper[5], hyper[6], hyper[7], dh[0], dh[1], masses.data(), corr, charges, r0, gate, parity};
  return mlip_model_create(&d, w.data(), count, precision, out);
}

int mlip_model_free(mlip_model* M) {
  if (!M) return MLIP_OK;
  cudaDeviceSynchronize();
  free_eval_graphs(M->egraph);
  M->egraph = nullptr;
  M->ws.release();
  if (M->d_weights) cudaFree(M->d_weights);
  if (M->d_w3img) cudaFree(M->d_w3img);
  if (M->d_wmixT) cudaFree(M->d_wmixT);
  if (M->d_gateT) cudaFree(M->d_gateT);
  if (M->d_miximg) cudaFree(M->d_miximg);
  if (M->d_gateimg) cudaFree(M->d_gateimg);
  if (M->d_gatescale) cudaFree(M->d_gatescale);
  if (M->d_radimg) cudaFree(M->d_radimg);
  if (M->d_embmax) cudaFree(M->d_embmax);
  if (M->d_mixscale) cudaFree(M->d_mixscale);
  delete M;
  return MLIP_OK;
}

int mlip_neighbors(const double* pos, int64_t n, const double cell[9], const uint8_t pbc[3], double cutoff,
                   int32_t* recv, int32_t* send, int8_t* shift, int64_t capacity, int64_t* n_edges,
                   int on_device, void* stream) {
  if (!n_edges || !cell || !pbc || (n > 0 && !pos)) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  *n_edges = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  static thread_local Workspace* ws = nullptr;
  if (!ws) ws = new Workspace();
  WsStream wss(*ws, st);
  const double* d_pos = pos;
  if (!on_device && n > 0) {
    double* dp = nullptr;
    MLIP_TRY(ws->get("in.pos", (size_t)3 * n, &dp));
    MLIP_CUDA_TRY(cudaMemcpyAsync(dp, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    d_pos = dp;
  }
  NeighborList nl;
  MLIP_TRY(build_neighbors(*ws, d_pos, n, cell, pbc, cutoff, false, st, &nl));
  *n_edges = nl.E;
  if (nl.E > capacity) { set_error("neighbour capacity %lld < %lld edges", (long long)capacity, (long long)nl.E); return MLIP_ERR_CAPACITY; }
  if (nl.E > 0) {
    if (!recv || !send || !shift) { set_error("null output buffer"); return MLIP_ERR_INVALID_ARG; }
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    MLIP_CUDA_TRY(cudaMemcpyAsync(recv, nl.recv, sizeof(int32_t) * nl.E, k, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(send, nl.send, sizeof(int32_t) * nl.E, k, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(shift, nl.shift, 3 * nl.E, k, st));
  }
  MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  return MLIP_OK;
}

}  // extern "C"

namespace mlip {

__global__ void check_inputs(int n, const double* __restrict__ pos, const int* __restrict__ species, int S,
                             int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int z = species[i];
  if (z < 0 || z >= S) atomicOr(flag, 1);
  if (!isfinite(pos[3 * i]) || !isfinite(pos[3 * i + 1]) || !isfinite(pos[3 * i + 2])) atomicOr(flag, 2);
}

int launch_check_inputs(int n, const double* pos, const int* species, int S, int* flag, cudaStream_t st) {
  if (n <= 0) return MLIP_OK;
  { MLIP_PROF("check_inputs", st); check_inputs<<<(n + 255) / 256, 256, 0, st>>>(n, pos, species, S, flag); }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}


int plain_forward_edges(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                        const NeighborList& nl, double* d_energy, cudaStream_t st) {
  Workspace& ws = M->ws;
  const int n = (int)b.n, C = M->C, D = M->D, T = M->T, L = M->L, H = M->H, P = M->P, P0 = M->P0;
  const float s = (float)(1.0 / M->avg_nb);
  const int E = (int)nl.E;
  const size_t Ec = (size_t)std::max(E, 1), ND = (size_t)std::max(n, 1) * D * C;

  CellArg ca{b.d_cell, b.d_sys_of, b.any_pbc() ? 1 : 0};

  float4 *ev = nullptr, *g = nullptr;
  float *z2T = nullptr, *m = nullptr, *Gm = nullptr, *Ga = nullptr, *Gb = nullptr, *dw = nullptr, *dz2 = nullptr,
        *dY = nullptr, *dr = nullptr;
  double* atom_e = nullptr;
  MLIP_TRY(ws.get("ef.ev", Ec, &ev));
  MLIP_TRY(ws.get("ef.g", Ec, &g));
  MLIP_TRY(ws.get("ef.z2T", Ec * H, &z2T));
  MLIP_TRY(ws.get("ef.m", ND, &m));
  MLIP_TRY(ws.get("ef.Gm", ND, &Gm));
  MLIP_TRY(ws.get("ef.Ga", ND, &Ga));
  MLIP_TRY(ws.get("ef.Gb", ND, &Gb));
  MLIP_TRY(ws.get("ef.dw", Ec * P * C, &dw));
  MLIP_TRY(ws.get("ef.dz2", Ec * H, &dz2));
  MLIP_TRY(ws.get("ef.dY", Ec * 16, &dY));
  MLIP_TRY(ws.get("ef.dr", Ec, &dr));
  MLIP_TRY(ws.get("ef.atom_e", (size_t)std::max(n, 1), &atom_e));
  std::vector<float*> h(T + 1), u0(T), w(T), A(T, nullptr), gpre(T, nullptr), gg(T, nullptr);
  for (int t = 0; t <= T; ++t) MLIP_TRY(ws.get("ef.h" + std::to_string(t), ND, &h[t]));
  for (int t = 0; t < T; ++t) {
    MLIP_TRY(ws.get("ef.u" + std::to_string(t), (size_t)n * C, &u0[t]));
    MLIP_TRY(ws.get("ef.w" + std::to_string(t), Ec * (t == 0 ? P0 : P) * C, &w[t]));
    if (M->corr == 2) MLIP_TRY(ws.get("ef.A" + std::to_string(t), ND, &A[t]));
    if (M->gate) {
      MLIP_TRY(ws.get("ef.gpre" + std::to_string(t), ND, &gpre[t]));
      MLIP_TRY(ws.get("ef.gg" + std::to_string(t), (size_t)std::max(n, 1) * L * C, &gg[t]));
    }
  }
  double* energy = d_energy;

  MLIP_TRY(launch_edge_geom(E, d_pos, nl.recv, nl.send, nl.shift, ca, ev, st));
  MLIP_TRY(launch_embed(n, C, D, M->S, d_species, M->W_emb, h[0], st));
  for (int t = 0; t < T; ++t) {
    const bool first = t == 0;
    const int PW = first ? P0 : P;
    MLIP_TRY(launch_radial_fwd(H, E, ev, M->W1[t], M->W2[t], (float)M->rc, M->p, z2T, E, st));
    MLIP_TRY(launch_sgemm(true, false, E, PW * C, H, z2T, E, M->W3[t], P * C, w[t], PW * C, st));
    MLIP_TRY(launch_tp_fwd(L, first, n, C, nl.row_ptr, nl.recv, nl.send, ev, h[t], w[t], PW, s, m, st, M->parity != 0));
    if (M->corr == 2)
      MLIP_TRY(launch_sym_contract(L, n, C, M->S, m, nullptr, d_species, M->Wsc1[t], M->Wsc2[t], A[t], m, st));
    if (M->gate)
      MLIP_TRY(launch_gate_fwd(L, n, C, M->S, d_species, m, nullptr, h[t], M->Wmix[t], M->Wself[t], M->Wgate[t],
                               M->Wselfgate[t], h[t + 1], gpre[t], gg[t], nullptr, nullptr, st));
    else
      MLIP_TRY(launch_mix_fwd(n, C, L, m, M->Wmix[t], h[t], h[t + 1], u0[t], st, M->parity));
  }
  if (M->charges) {  // readout, charge head and Coulomb term, then the per-system sums
    MLIP_TRY(launch_readout(n, C, D, M->S, d_species, M->W_out, M->E0, h[T], atom_e, st));
    MLIP_TRY(coulomb_forward(ws, b, M, d_pos, d_species, h[T], atom_e, st));
    MLIP_TRY(launch_seg_sum(ws, b, 1, atom_e, false, energy, st));
  } else {
    MLIP_TRY(launch_energy(ws, b, C, D, M->S, d_species, M->W_out, M->E0, h[T], atom_e, energy, st));
  }
  return MLIP_OK;
}

int plain_adjoint_edges(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                        const NeighborList& nl, double* d_forces, double* d_stress, cudaStream_t st) {
  Workspace& ws = M->ws;
  const int n = (int)b.n, C = M->C, D = M->D, T = M->T, L = M->L, H = M->H, P = M->P, P0 = M->P0;
  const float s = (float)(1.0 / M->avg_nb);
  const int E = (int)nl.E;
  const size_t Ec = (size_t)std::max(E, 1), ND = (size_t)std::max(n, 1) * D * C;

  CellArg ca{b.d_cell, b.d_sys_of, b.any_pbc() ? 1 : 0};

  float4 *ev = nullptr, *g = nullptr;
  float *z2T = nullptr, *m = nullptr, *Gm = nullptr, *Ga = nullptr, *Gb = nullptr, *dw = nullptr, *dz2 = nullptr,
        *dY = nullptr, *dr = nullptr;
  double* atom_e = nullptr;
  MLIP_TRY(ws.get("ef.ev", Ec, &ev));
  MLIP_TRY(ws.get("ef.g", Ec, &g));
  MLIP_TRY(ws.get("ef.z2T", Ec * H, &z2T));
  MLIP_TRY(ws.get("ef.m", ND, &m));
  MLIP_TRY(ws.get("ef.Gm", ND, &Gm));
  MLIP_TRY(ws.get("ef.Ga", ND, &Ga));
  MLIP_TRY(ws.get("ef.Gb", ND, &Gb));
  MLIP_TRY(ws.get("ef.dw", Ec * P * C, &dw));
  MLIP_TRY(ws.get("ef.dz2", Ec * H, &dz2));
  MLIP_TRY(ws.get("ef.dY", Ec * 16, &dY));
  MLIP_TRY(ws.get("ef.dr", Ec, &dr));
  MLIP_TRY(ws.get("ef.atom_e", (size_t)std::max(n, 1), &atom_e));
  std::vector<float*> h(T + 1), u0(T), w(T), A(T, nullptr), gpre(T, nullptr), gg(T, nullptr);
  for (int t = 0; t <= T; ++t) MLIP_TRY(ws.get("ef.h" + std::to_string(t), ND, &h[t]));
  for (int t = 0; t < T; ++t) {
    MLIP_TRY(ws.get("ef.u" + std::to_string(t), (size_t)n * C, &u0[t]));
    MLIP_TRY(ws.get("ef.w" + std::to_string(t), Ec * (t == 0 ? P0 : P) * C, &w[t]));
    if (M->corr == 2) MLIP_TRY(ws.get("ef.A" + std::to_string(t), ND, &A[t]));
    if (M->gate) {
      MLIP_TRY(ws.get("ef.gpre" + std::to_string(t), ND, &gpre[t]));
      MLIP_TRY(ws.get("ef.gg" + std::to_string(t), (size_t)std::max(n, 1) * L * C, &gg[t]));
    }
  }
  {
    MLIP_TRY(launch_grad_init(n, C, D, M->S, d_species, M->W_out, Ga, st));
    if (M->charges) MLIP_TRY(coulomb_adjoint(ws, b, M, d_species, Ga, st));
    MLIP_CUDA_TRY(cudaMemsetAsync(dY, 0, Ec * 16 * sizeof(float), st));
    MLIP_CUDA_TRY(cudaMemsetAsync(dr, 0, Ec * sizeof(float), st));
    for (int t = T - 1; t >= 0; --t) {
      const bool first = t == 0;
      const int PW = first ? P0 : P;
      if (M->gate)  // Gm = dE/dm; Ga becomes dE/dh^t's residual part (with the self-connection)
        MLIP_TRY(launch_gate_bwd(L, n, C, M->S, d_species, Ga, nullptr, gpre[t], gg[t], M->WmixT[t], M->WselfT[t],
                                 M->WgateT[t], M->WselfgateT[t], Gm, nullptr, nullptr, st));
      else
        MLIP_TRY(launch_mix_bwd(n, C, L, Ga, u0[t], M->Wmix[t], M->WmixT[t], Gm, st, M->parity));
      if (M->corr == 2)
        MLIP_TRY(launch_sym_contract_bwd(L, n, C, M->S, Gm, A[t], d_species, M->Wsc1[t], M->Wsc2[t], Gm, nullptr, nullptr,
                                         st));
      MLIP_TRY(launch_tp_bwd(L, first, n, C, nl.row_ptr, nl.recv, nl.send, ev, h[t], Gm, w[t], PW, s, Ga, Gb, dw, dY, st,
                             M->parity != 0));
      MLIP_TRY(launch_sgemm(false, true, E, H, PW * C, dw, PW * C, M->W3[t], P * C, dz2, H, st));
      MLIP_TRY(launch_radial_bwd(H, E, ev, M->W1[t], M->W2[t], (float)M->rc, M->p, dz2, dr, st));
      std::swap(Ga, Gb);
    }
    MLIP_TRY(launch_edge_grad(E, ev, dY, dr, g, st));
    double* fbuf = d_forces;
    if (!fbuf) MLIP_TRY(ws.get("ef.fscratch", (size_t)3 * std::max(n, 1), &fbuf));
    MLIP_TRY(launch_forces_virial(ws, b, nl.row_ptr, nl.rev, g, ev, fbuf, d_stress, st));
    if (M->charges) MLIP_TRY(coulomb_add_forces(ws, b, fbuf, st));
  }
  return MLIP_OK;
}

int evaluate_plain(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                   double* d_energy, double* d_forces, double* d_stress, cudaStream_t st) {
  Workspace& ws = M->ws;
  int* flag = nullptr;
  MLIP_TRY(ws.get("chk.flag", 1, &flag));
  MLIP_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
  MLIP_TRY(launch_check_inputs((int)b.n, d_pos, d_species, M->S, flag, st));
  NeighborList nl;
  MLIP_TRY(build_neighbors_batch(ws, d_pos, b, M->rc, true, st, &nl));
  int hflag = 0;
  MLIP_CUDA_TRY(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  if (hflag & 1) { set_error("species index out of range"); return MLIP_ERR_INVALID_ARG; }
  if (hflag & 2) { set_error("non-finite position"); return MLIP_ERR_INVALID_ARG; }
  MLIP_TRY(plain_forward_edges(M, d_pos, d_species, b, nl, d_energy, st));
  if (d_forces || d_stress) MLIP_TRY(plain_adjoint_edges(M, d_pos, d_species, b, nl, d_forces, d_stress, st));
  return MLIP_OK;
}

int evaluate(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b, double* d_energy,
             double* d_forces, double* d_stress, cudaStream_t st, bool graph) {
  ++M->eval_gen;  // the workspace is written: a saved separate forward is no longer usable
  if (M->charges && b.any_pbc()) {
    set_error("a model with charges evaluates open systems only (the Coulomb term has no periodic images)");
    return MLIP_ERR_CELL;
  }
  if (M->precision == MLIP_PREC_FP32) return evaluate_plain(M, d_pos, d_species, b, d_energy, d_forces, d_stress, st);
  if (graph) return evaluate_fused_graph(M, d_pos, d_species, b, d_energy, d_forces, d_stress, st);
  return evaluate_fused(M, d_pos, d_species, b, d_energy, d_forces, d_stress, st);
}

}  // namespace mlip

extern "C" int mlip_energy_forces(mlip_model* M, const double* pos, const int32_t* species, int64_t n,
                                  const double cell[9], const uint8_t pbc[3], double* energy, double* forces,
                                  double* stress, int on_device, void* stream) {
  using namespace mlip;
  if (!M || !pos || !species || !energy || !cell || !pbc) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  if (n < 1 || n > (1LL << 28)) { set_error("atom count %lld out of range", (long long)n); return MLIP_ERR_INVALID_ARG; }
  if (stress && !(pbc[0] && pbc[1] && pbc[2])) { set_error("stress needs a fully periodic cell"); return MLIP_ERR_CELL; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != M->device) { set_error("model lives on device %d, current device is %d", M->device, cur); return MLIP_ERR_INVALID_ARG; }
  Workspace& ws = M->ws;
  WsStream wss(ws, st);
  const double* d_pos = pos;
  const int* d_species = species;
  double *d_energy = energy, *d_forces = forces, *d_stress = stress;
  if (!on_device) {
    if (!(pbc[0] || pbc[1] || pbc[2])) { /* cell ignored */ }
    for (int64_t i = 0; i < n; ++i)
      if (species[i] < 0 || species[i] >= M->S) { set_error("species[%lld] = %d out of range", (long long)i, species[i]); return MLIP_ERR_INVALID_ARG; }
    double* dp = nullptr;
    int* dz = nullptr;
    MLIP_TRY(ws.get("in.pos", (size_t)3 * n, &dp));
    MLIP_TRY(ws.get("in.species", (size_t)n, &dz));
    MLIP_TRY(ws.get("out.energy", 1, &d_energy));
    if (forces) MLIP_TRY(ws.get("out.forces", (size_t)3 * n, &d_forces));
    if (stress) MLIP_TRY(ws.get("out.stress", 9, &d_stress));
    MLIP_CUDA_TRY(cudaMemcpyAsync(dp, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(dz, species, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    d_pos = dp;
    d_species = dz;
  }
  SystemBatch b;
  single_system(b, n, cell, pbc);
  MLIP_TRY(upload_batch(ws, M->stage, b, st));
  MLIP_TRY(evaluate(M, d_pos, d_species, b, d_energy, d_forces, d_stress, st, true));
  if (!on_device) {
    MLIP_CUDA_TRY(cudaMemcpyAsync(energy, d_energy, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (forces) MLIP_CUDA_TRY(cudaMemcpyAsync(forces, d_forces, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    if (stress) MLIP_CUDA_TRY(cudaMemcpyAsync(stress, d_stress, sizeof(double) * 9, cudaMemcpyDeviceToHost, st));
    MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  } else {
    MLIP_CUDA_TRY(cudaGetLastError());
  }
  return MLIP_OK;
}

namespace mlip {
// out[k] = -g F[k] = g dE/dr_k (the gradient of g E with respect to the positions)
__global__ void grad_from_forces(int64_t n3, const double* __restrict__ F, const double* __restrict__ g,
                                 double* __restrict__ out) {
  const double gv = *g;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = -gv * F[k];
}
// out[k] = g s[k] (9 stress components)
__global__ void scale_stress(const double* __restrict__ S, const double* __restrict__ g, double* __restrict__ out) {
  if (threadIdx.x < 9) out[threadIdx.x] = *g * S[threadIdx.x];
}
}  // namespace mlip

extern "C" int mlip_energy_forward(mlip_model* M, const double* pos, const int32_t* species, int64_t n,
                                   const double cell[9], const uint8_t pbc[3], double* energy, int on_device,
                                   void* stream) {
  using namespace mlip;
  if (!M || !pos || !species || !energy || !cell || !pbc) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  if (n < 1 || n > (1LL << 28)) { set_error("atom count %lld out of range", (long long)n); return MLIP_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != M->device) { set_error("model lives on device %d, current device is %d", M->device, cur); return MLIP_ERR_INVALID_ARG; }
  Workspace& ws = M->ws;
  WsStream wss(ws, st);
  ++M->eval_gen;
  M->tape_gen = 0;
  // the library's own copies of the inputs, which the backward reads
  double* d_pos = nullptr;
  int* d_sp = nullptr;
  double* d_energy = nullptr;
  int* flag = nullptr;
  MLIP_TRY(ws.get("tape.pos", (size_t)3 * n, &d_pos));
  MLIP_TRY(ws.get("tape.species", (size_t)n, &d_sp));
  MLIP_TRY(ws.get("tape.energy", 1, &d_energy));
  MLIP_TRY(ws.get("chk.flag", 2, &flag));
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  MLIP_CUDA_TRY(cudaMemcpyAsync(d_pos, pos, sizeof(double) * 3 * n, k, st));
  MLIP_CUDA_TRY(cudaMemcpyAsync(d_sp, species, sizeof(int) * n, k, st));
  SystemBatch& b = M->tape_batch;
  b = SystemBatch();
  single_system(b, n, cell, pbc);
  MLIP_TRY(upload_batch(ws, M->stage, b, st));
  // inputs are checked before any kernel reads a weight row by species
  MLIP_CUDA_TRY(cudaMemsetAsync(flag, 0, 2 * sizeof(int), st));
  MLIP_TRY(launch_check_inputs((int)n, d_pos, d_sp, M->S, flag, st));
  NeighborList nl;
  MLIP_TRY(build_neighbors_batch(ws, d_pos, b, M->rc, true, st, &nl));
  MLIP_TRY(check_eval_flags(flag, st));
  if (M->charges && b.any_pbc()) {
    set_error("a model with charges evaluates open systems only (the Coulomb term has no periodic images)");
    return MLIP_ERR_CELL;
  }
  if (M->precision == MLIP_PREC_FP32) {
    MLIP_TRY(plain_forward_edges(M, d_pos, d_sp, b, nl, d_energy, st));
  } else {
    MLIP_TRY(fused_forward_edges(M, d_pos, d_sp, b, nl, nullptr, flag, d_energy, st));
    MLIP_TRY(check_eval_flags(flag, st));
  }
  M->tape_nl = nl;
  M->tape_gen = M->eval_gen;
  MLIP_CUDA_TRY(cudaMemcpyAsync(energy, d_energy, sizeof(double),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  if (!on_device) MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  return MLIP_OK;
}

extern "C" int mlip_energy_backward(mlip_model* M, const double* grad_energy, double* grad_pos, double* stress,
                                    int on_device, void* stream) {
  using namespace mlip;
  if (!M || !grad_energy || !grad_pos) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  if (M->tape_gen == 0 || M->tape_gen != M->eval_gen) {
    set_error("no saved forward to differentiate: call mlip_energy_forward first (any other evaluation of the "
              "model in between overwrites it)");
    return MLIP_ERR_INVALID_ARG;
  }
  const SystemBatch& b = M->tape_batch;
  const int64_t n = b.n;
  if (stress && !(b.pbc[0] && b.pbc[1] && b.pbc[2])) { set_error("stress needs a fully periodic cell"); return MLIP_ERR_CELL; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != M->device) { set_error("model lives on device %d, current device is %d", M->device, cur); return MLIP_ERR_INVALID_ARG; }
  Workspace& ws = M->ws;
  WsStream wss(ws, st);
  double *d_pos = nullptr, *d_F = nullptr, *d_S = nullptr, *d_g = nullptr, *d_out = grad_pos, *d_sout = stress;
  int* d_sp = nullptr;
  int* flag = nullptr;
  MLIP_TRY(ws.get("tape.pos", (size_t)3 * n, &d_pos));
  MLIP_TRY(ws.get("tape.species", (size_t)n, &d_sp));
  MLIP_TRY(ws.get("tape.forces", (size_t)3 * n, &d_F));
  if (stress) MLIP_TRY(ws.get("tape.stress", 9, &d_S));
  MLIP_TRY(ws.get("chk.flag", 2, &flag));
  if (on_device) {
    d_g = const_cast<double*>(grad_energy);
  } else {
    MLIP_TRY(ws.get("tape.grad", 1, &d_g));
    MLIP_TRY(ws.get("tape.grad_pos", (size_t)3 * n, &d_out));
    if (stress) MLIP_TRY(ws.get("tape.grad_stress", 9, &d_sout));
    MLIP_CUDA_TRY(cudaMemcpyAsync(d_g, grad_energy, sizeof(double), cudaMemcpyHostToDevice, st));
  }
  if (M->precision == MLIP_PREC_FP32) {
    MLIP_TRY(plain_adjoint_edges(M, d_pos, d_sp, b, M->tape_nl, d_F, d_S, st));
  } else {
    MLIP_CUDA_TRY(cudaMemsetAsync(flag, 0, 2 * sizeof(int), st));
    MLIP_TRY(fused_adjoint_edges(M, d_pos, d_sp, b, M->tape_nl, nullptr, flag, d_F, d_S, true, st));
  }
  {
    MLIP_PROF("grad_from_forces", st);
    const int64_t n3 = 3 * n;
    grad_from_forces<<<(int)std::min<int64_t>((n3 + 255) / 256, 4096), 256, 0, st>>>(n3, d_F, d_g, d_out);
  }
  if (stress) {
    MLIP_PROF("scale_stress", st);
    scale_stress<<<1, 32, 0, st>>>(d_S, d_g, d_sout);
  }
  MLIP_LAUNCH_CHECK();
  if (M->precision != MLIP_PREC_FP32) MLIP_TRY(check_eval_flags(flag, st));
  if (!on_device) {
    MLIP_CUDA_TRY(cudaMemcpyAsync(grad_pos, d_out, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    if (stress) MLIP_CUDA_TRY(cudaMemcpyAsync(stress, d_sout, sizeof(double) * 9, cudaMemcpyDeviceToHost, st));
    MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  }
  return MLIP_OK;
}

extern "C" int mlip_energy_forces_charged(mlip_model* M, const double* pos, const int32_t* species, int64_t n,
                                          double total_charge, double* energy, double* forces, double* charges,
                                          int on_device, void* stream) {
  using namespace mlip;
  if (!M || !pos || !species || !energy) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  if (!M->charges) { set_error("the model has no charge head (charges = 0)"); return MLIP_ERR_INVALID_ARG; }
  if (n < 1 || n > (1LL << 28)) { set_error("atom count %lld out of range", (long long)n); return MLIP_ERR_INVALID_ARG; }
  if (!std::isfinite(total_charge)) { set_error("total charge is not finite"); return MLIP_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != M->device) { set_error("model lives on device %d, current device is %d", M->device, cur); return MLIP_ERR_INVALID_ARG; }
  Workspace& ws = M->ws;
  WsStream wss(ws, st);
  const double* d_pos = pos;
  const int* d_species = species;
  double *d_energy = energy, *d_forces = forces;
  if (!on_device) {
    for (int64_t i = 0; i < n; ++i)
      if (species[i] < 0 || species[i] >= M->S) { set_error("species[%lld] = %d out of range", (long long)i, species[i]); return MLIP_ERR_INVALID_ARG; }
    double* dp = nullptr;
    int* dz = nullptr;
    MLIP_TRY(ws.get("in.pos", (size_t)3 * n, &dp));
    MLIP_TRY(ws.get("in.species", (size_t)n, &dz));
    MLIP_TRY(ws.get("out.energy", 1, &d_energy));
    if (forces) MLIP_TRY(ws.get("out.forces", (size_t)3 * n, &d_forces));
    MLIP_CUDA_TRY(cudaMemcpyAsync(dp, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(dz, species, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    d_pos = dp;
    d_species = dz;
  }
  const double cell[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const uint8_t pbc[3] = {0, 0, 0};
  SystemBatch b;
  single_system(b, n, cell, pbc);
  b.qtot.assign(1, total_charge);
  MLIP_TRY(upload_batch(ws, M->stage, b, st));
  MLIP_TRY(evaluate(M, d_pos, d_species, b, d_energy, d_forces, nullptr, st, true));
  double* d_q = nullptr;
  MLIP_TRY(coulomb_charges(ws, b, &d_q));
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (charges) MLIP_CUDA_TRY(cudaMemcpyAsync(charges, d_q, sizeof(double) * n, k, st));
  if (!on_device) {
    MLIP_CUDA_TRY(cudaMemcpyAsync(energy, d_energy, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (forces) MLIP_CUDA_TRY(cudaMemcpyAsync(forces, d_forces, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  } else {
    MLIP_CUDA_TRY(cudaGetLastError());
  }
  return MLIP_OK;
}

extern "C" int mlip_energy_forces_batch(mlip_model* M, int32_t n_systems, const int64_t* atom_off, const double* pos,
                                        const int32_t* species, const double* cells, const uint8_t* pbc,
                                        double* energy, double* forces, double* stress, int on_device,
                                        void* stream) {
  using namespace mlip;
  if (!M || !atom_off || !pos || !species || !cells || !pbc || !energy) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  if (n_systems < 1 || n_systems > (1 << 20)) { set_error("system count %d out of range", n_systems); return MLIP_ERR_INVALID_ARG; }
  if (atom_off[0] != 0) { set_error("atom_off[0] must be 0"); return MLIP_ERR_INVALID_ARG; }
  for (int s = 0; s < n_systems; ++s) {
    if (atom_off[s + 1] <= atom_off[s]) { set_error("system %d has no atoms (atom_off must increase)", s); return MLIP_ERR_INVALID_ARG; }
    if (stress && !(pbc[3 * s] && pbc[3 * s + 1] && pbc[3 * s + 2])) {
      set_error("stress needs a fully periodic cell (system %d)", s);
      return MLIP_ERR_CELL;
    }
  }
  const int64_t n = atom_off[n_systems];
  if (n > (1LL << 28)) { set_error("atom count %lld out of range", (long long)n); return MLIP_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != M->device) { set_error("model lives on device %d, current device is %d", M->device, cur); return MLIP_ERR_INVALID_ARG; }
  Workspace& ws = M->ws;
  WsStream wss(ws, st);
  const double* d_pos = pos;
  const int* d_species = species;
  double *d_energy = energy, *d_forces = forces, *d_stress = stress;
  if (!on_device) {
    for (int64_t i = 0; i < n; ++i)
      if (species[i] < 0 || species[i] >= M->S) { set_error("species[%lld] = %d out of range", (long long)i, species[i]); return MLIP_ERR_INVALID_ARG; }
    double* dp = nullptr;
    int* dz = nullptr;
    MLIP_TRY(ws.get("in.pos", (size_t)3 * n, &dp));
    MLIP_TRY(ws.get("in.species", (size_t)n, &dz));
    MLIP_TRY(ws.get("out.energy", (size_t)n_systems, &d_energy));
    if (forces) MLIP_TRY(ws.get("out.forces", (size_t)3 * n, &d_forces));
    if (stress) MLIP_TRY(ws.get("out.stress", (size_t)9 * n_systems, &d_stress));
    MLIP_CUDA_TRY(cudaMemcpyAsync(dp, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(dz, species, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    d_pos = dp;
    d_species = dz;
  }
  SystemBatch b;
  b.nsys = n_systems;
  b.atom_off.assign(atom_off, atom_off + n_systems + 1);
  b.cell.assign(cells, cells + 9 * (size_t)n_systems);
  b.pbc.assign(pbc, pbc + 3 * (size_t)n_systems);
  MLIP_TRY(upload_batch(ws, M->stage, b, st));
  MLIP_TRY(evaluate(M, d_pos, d_species, b, d_energy, d_forces, d_stress, st, true));
  if (!on_device) {
    MLIP_CUDA_TRY(cudaMemcpyAsync(energy, d_energy, sizeof(double) * n_systems, cudaMemcpyDeviceToHost, st));
    if (forces) MLIP_CUDA_TRY(cudaMemcpyAsync(forces, d_forces, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    if (stress) MLIP_CUDA_TRY(cudaMemcpyAsync(stress, d_stress, sizeof(double) * 9 * n_systems, cudaMemcpyDeviceToHost, st));
    MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  } else {
    MLIP_CUDA_TRY(cudaGetLastError());
  }
  return MLIP_OK;
}
