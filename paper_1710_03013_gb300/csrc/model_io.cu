// kkm_model_save / kkm_model_load: a fitted model to and from a file, so that
// a resident model survives a restart of the serving process.  The paper has
// no persistence; the state kept is what kkm_assign / kkm_cost and the model
// queries read (the last mini-batch's landmark supports with their sorted
// structure and g_hat, the global medoids and counts, the trace).
//
// Format (little-endian): 8-byte magic "KKMMOD02", then int64 C, d, kind,
// n_atoms, dp, nL, max_units, trace length T, a float64 sigma, then the
// arrays in a fixed order, each exactly as many bytes as its element count
// implies, then int64 D and the D float64 centre displacements (files of the
// first version, magic "KKMMOD01", end before D and load with none).
// Loading checks every count against the header (and the file length
// against their sum) before it touches the GPU.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <memory>
#include <string>
#include <vector>

#include "internal.h"

namespace kkm {

static const char kMagic[8] = {'K', 'K', 'M', 'M', 'O', 'D', '0', '2'};
static const char kMagicV1[8] = {'K', 'K', 'M', 'M', 'O', 'D', '0', '1'};

struct Header {
  int64_t C, d, kind, n_atoms, dp, nL, max_units, T;
  double sigma;
};

static int64_t expected_dp(const Header& h) {
  if (h.kind == KKM_RMSD) return 3 * round_up(h.n_atoms, 8);
  return round_up(h.d, 8);
}

// Bytes of the array part for a header.
static int64_t body_bytes(const Header& h) {
  const int64_t C = h.C, nL = h.nL, dp = h.dp, mu = h.max_units, T = h.T, d = h.d;
  int64_t b = 0;
  b += nL * dp * 4 + nL * 4 + nL * 8 + nL * 4 + nL * 4 + nL * 4;  // sup, sup_aux, ids, labels, L_ident, perm
  b += (C + 1) * 4 + C * 4 + 3 * mu * 4 + (C + 1) * 4 + 4;          // seg_off, n_j, units, seg_unit, n_units
  b += C * 8 + C * dp * 4 + C * 4;                                  // ghat, med, med_aux
  b += C * 8 + C * 8 + T * 8 + T * 4;                               // medoids, W, omega, changed
  b += nL * 4 + C * 8 + C * 4 + C * d * 4;                          // host copies: labels, ghat, n, coords
  return b;
}

struct Io {
  FILE* f;
  bool ok = true;
  void put(const void* p, size_t n) {
    if (ok && n && fwrite(p, 1, n, f) != n) ok = false;
  }
  void get(void* p, size_t n) {
    if (ok && n && fread(p, 1, n, f) != n) ok = false;
  }
};

static kkm_status fail(const std::string& msg) {
  set_error(msg);
  return KKM_EINVAL;
}

static kkm_status save_impl(const kkm_model* m, const char* path) {
  if (!m || !path) return fail("model and path must not be NULL");
  Header h{m->C, m->d, m->kind, m->n_atoms, m->dp, m->nL, m->max_units, (int64_t)m->omega.size(), (double)m->sigma};
  // device arrays to the host first (the file is written only if all copies succeed)
  std::vector<unsigned char> dev((size_t)(body_bytes(h)));
  size_t off = 0;
  auto D = [&](const void* src, size_t bytes) -> kkm_status {
    KKM_CK(cudaMemcpy(dev.data() + off, src, bytes, cudaMemcpyDeviceToHost));
    off += bytes;
    return KKM_OK;
  };
  const int64_t C = h.C, nL = h.nL, dp = h.dp, mu = h.max_units;
  KKM_TRY(D(m->sup, (size_t)(nL * dp * 4)));
  KKM_TRY(D(m->sup_aux, (size_t)nL * 4));
  KKM_TRY(D(m->sup_ids, (size_t)nL * 8));
  KKM_TRY(D(m->sup_labels, (size_t)nL * 4));
  KKM_TRY(D(m->L_ident, (size_t)nL * 4));
  KKM_TRY(D(m->perm, (size_t)nL * 4));
  KKM_TRY(D(m->seg_off, (size_t)(C + 1) * 4));
  KKM_TRY(D(m->n_j, (size_t)C * 4));
  KKM_TRY(D(m->unit_j, (size_t)mu * 4));
  KKM_TRY(D(m->unit_kb, (size_t)mu * 4));
  KKM_TRY(D(m->unit_ke, (size_t)mu * 4));
  KKM_TRY(D(m->seg_unit, (size_t)(C + 1) * 4));
  KKM_TRY(D(m->n_units, 4));
  KKM_TRY(D(m->ghat, (size_t)C * 8));
  KKM_TRY(D(m->med, (size_t)(C * dp * 4)));
  KKM_TRY(D(m->med_aux, (size_t)C * 4));
  FILE* f = fopen(path, "wb");
  if (!f) return fail(std::string("cannot open ") + path + " for writing");
  Io io{f};
  io.put(kMagic, 8);
  io.put(&h, sizeof(h));
  io.put(dev.data(), off);
  io.put(m->medoids.data(), m->medoids.size() * 8);
  io.put(m->W.data(), m->W.size() * 8);
  io.put(m->omega.data(), m->omega.size() * 8);
  io.put(m->changed.data(), m->changed.size() * 4);
  io.put(m->sup_labels_h.data(), m->sup_labels_h.size() * 4);
  io.put(m->ghat_h.data(), m->ghat_h.size() * 8);
  io.put(m->n_h.data(), m->n_h.size() * 4);
  io.put(m->med_coords_h.data(), m->med_coords_h.size() * 4);
  const int64_t nd = (int64_t)m->displacement.size();
  io.put(&nd, 8);
  io.put(m->displacement.data(), (size_t)nd * 8);
  const bool ok = io.ok && fclose(f) == 0;
  if (!ok) return fail(std::string("write to ") + path + " failed");
  return KKM_OK;
}

static kkm_status load_impl(const char* path, kkm_model** out) {
  if (!path || !out) return fail("path and out must not be NULL");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return fail(std::string("cannot open ") + path);
  Io io{f};
  char magic[8];
  Header h;
  io.get(magic, 8);
  io.get(&h, sizeof(h));
  fseek(f, 0, SEEK_END);
  const long fsize = ftell(f);
  const bool v2 = io.ok && memcmp(magic, kMagic, 8) == 0;
  if (!io.ok || (!v2 && memcmp(magic, kMagicV1, 8) != 0)) {
    fclose(f);
    return fail(std::string(path) + " is not a kkm model file");
  }
  const bool sane = h.C >= 1 && h.C <= kMaxC && h.d >= 1 && h.d <= (1 << 24) && h.nL >= 1 && h.nL <= (1 << 28) &&
                    (h.kind == KKM_RBF || h.kind == KKM_RMSD || h.kind == KKM_LINEAR) &&
                    (h.kind != KKM_RMSD || (h.n_atoms >= 1 && h.d == 3 * h.n_atoms)) && h.dp == expected_dp(h) &&
                    h.max_units == max_units_for((int)h.nL, (int)h.C) && h.T >= 0 && h.T <= (1 << 28) &&
                    h.sigma == h.sigma;
  const long base = sane ? (long)(8 + sizeof(Header) + body_bytes(h)) : 0;
  int64_t nd = 0;
  if (sane && v2) {  // the displacement count follows the arrays
    fseek(f, base, SEEK_SET);
    io.get(&nd, 8);
  }
  const bool nd_ok = io.ok && nd >= 0 && nd <= (1 << 24);
  if (!sane || !nd_ok || fsize != base + (v2 ? (long)(8 + 8 * nd) : 0L)) {
    fclose(f);
    return fail(std::string(path) + ": inconsistent model header or file length");
  }
  fseek(f, (long)(8 + sizeof(Header)), SEEK_SET);
  auto* m = new kkm_model();
  std::unique_ptr<kkm_model> guard(m);
  m->C = (int)h.C;
  m->d = h.d;
  m->kind = (int)h.kind;
  m->sigma = (float)h.sigma;
  m->n_atoms = (int)h.n_atoms;
  m->dp = (int)h.dp;
  m->nL = (int)h.nL;
  m->max_units = (int)h.max_units;
  KKM_CK(cudaGetDevice(&m->device));
  const int64_t C = h.C, nL = h.nL, dp = h.dp, mu = h.max_units;
  std::vector<unsigned char> buf;
  auto H2D = [&](void* dst, size_t bytes) -> kkm_status {
    buf.resize(bytes);
    io.get(buf.data(), bytes);
    if (!io.ok) return fail(std::string(path) + ": truncated");
    KKM_CK(cudaMemcpy(dst, buf.data(), bytes, cudaMemcpyHostToDevice));
    return KKM_OK;
  };
  kkm_status st = model_alloc_device(m);
  if (st != KKM_OK) {
    fclose(f);
    return st;
  }
  kkm_status r = KKM_OK;
  auto step = [&](kkm_status s) {
    if (r == KKM_OK) r = s;
  };
  step(H2D(m->sup, (size_t)(nL * dp * 4)));
  step(H2D(m->sup_aux, (size_t)nL * 4));
  step(H2D(m->sup_ids, (size_t)nL * 8));
  step(H2D(m->sup_labels, (size_t)nL * 4));
  step(H2D(m->L_ident, (size_t)nL * 4));
  step(H2D(m->perm, (size_t)nL * 4));
  step(H2D(m->seg_off, (size_t)(C + 1) * 4));
  step(H2D(m->n_j, (size_t)C * 4));
  step(H2D(m->unit_j, (size_t)mu * 4));
  step(H2D(m->unit_kb, (size_t)mu * 4));
  step(H2D(m->unit_ke, (size_t)mu * 4));
  step(H2D(m->seg_unit, (size_t)(C + 1) * 4));
  step(H2D(m->n_units, 4));
  step(H2D(m->ghat, (size_t)C * 8));
  step(H2D(m->med, (size_t)(C * dp * 4)));
  step(H2D(m->med_aux, (size_t)C * 4));
  m->medoids.resize(C);
  m->W.resize(C);
  m->omega.resize(h.T);
  m->changed.resize(h.T);
  m->sup_labels_h.resize(nL);
  m->ghat_h.resize(C);
  m->n_h.resize(C);
  m->med_coords_h.resize((size_t)(C * h.d));
  io.get(m->medoids.data(), (size_t)C * 8);
  io.get(m->W.data(), (size_t)C * 8);
  io.get(m->omega.data(), (size_t)h.T * 8);
  io.get(m->changed.data(), (size_t)h.T * 4);
  io.get(m->sup_labels_h.data(), (size_t)nL * 4);
  io.get(m->ghat_h.data(), (size_t)C * 8);
  io.get(m->n_h.data(), (size_t)C * 4);
  io.get(m->med_coords_h.data(), (size_t)(C * h.d) * 4);
  if (v2) {
    int64_t nd2 = 0;
    io.get(&nd2, 8);
    m->displacement.resize((size_t)nd);
    io.get(m->displacement.data(), (size_t)nd * 8);
  }
  fclose(f);
  if (r != KKM_OK) return r;
  if (!io.ok) return fail(std::string(path) + ": truncated");
  *out = guard.release();
  return KKM_OK;
}

// ---------------------------------------------------------------------------
// Checkpoints of a fit between mini-batches (kkm_fit_range).  Format
// (little-endian): magic "KKMCKP01"; int64 N, d; int32 C, B; float64 s;
// int32 kind, n_atoms, iters; float32 sigma_arg; uint64 seed; int32
// precision, sampling, early_stop, had_init, next_batch; float32 sigma;
// int64 T; then int64 M[C], int64 W[C], float64 omega[T], int32 changed[T],
// float64 displacement[next_batch].  Every field is written on its own, so
// the layout does not depend on structure padding.
static const char kCkptMagic[8] = {'K', 'K', 'M', 'C', 'K', 'P', '0', '1'};

static kkm_status ckpt_save_impl(const kkm_checkpoint* c, const char* path) {
  if (!c || !path) return fail("checkpoint and path must not be NULL");
  FILE* f = fopen(path, "wb");
  if (!f) return fail(std::string("cannot open ") + path + " for writing");
  Io io{f};
  const int64_t T = (int64_t)c->omega.size();
  io.put(kCkptMagic, 8);
  io.put(&c->N, 8);
  io.put(&c->d, 8);
  io.put(&c->C, 4);
  io.put(&c->B, 4);
  io.put(&c->s, 8);
  io.put(&c->kind, 4);
  io.put(&c->n_atoms, 4);
  io.put(&c->iters, 4);
  io.put(&c->sigma_arg, 4);
  io.put(&c->seed, 8);
  io.put(&c->precision, 4);
  io.put(&c->sampling, 4);
  io.put(&c->early_stop, 4);
  io.put(&c->had_init, 4);
  io.put(&c->next_batch, 4);
  io.put(&c->sigma, 4);
  io.put(&T, 8);
  io.put(c->M.data(), c->M.size() * 8);
  io.put(c->W.data(), c->W.size() * 8);
  io.put(c->omega.data(), (size_t)T * 8);
  io.put(c->changed.data(), (size_t)T * 4);
  io.put(c->displacement.data(), c->displacement.size() * 8);
  const bool closed = fclose(f) == 0;
  if (!io.ok || !closed) return fail(std::string(path) + ": write failed");
  return KKM_OK;
}

static kkm_status ckpt_load_impl(const char* path, kkm_checkpoint** out) {
  if (!path || !out) return fail("path and out must not be NULL");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return fail(std::string("cannot open ") + path);
  std::unique_ptr<FILE, int (*)(FILE*)> fguard(f, fclose);
  fseek(f, 0, SEEK_END);
  const long len = ftell(f);
  fseek(f, 0, SEEK_SET);
  Io io{f};
  char magic[8] = {0};
  io.get(magic, 8);
  if (!io.ok || memcmp(magic, kCkptMagic, 8) != 0) return fail(std::string(path) + ": not a kkm checkpoint");
  std::unique_ptr<kkm_checkpoint> c(new kkm_checkpoint());
  int64_t T = 0;
  io.get(&c->N, 8);
  io.get(&c->d, 8);
  io.get(&c->C, 4);
  io.get(&c->B, 4);
  io.get(&c->s, 8);
  io.get(&c->kind, 4);
  io.get(&c->n_atoms, 4);
  io.get(&c->iters, 4);
  io.get(&c->sigma_arg, 4);
  io.get(&c->seed, 8);
  io.get(&c->precision, 4);
  io.get(&c->sampling, 4);
  io.get(&c->early_stop, 4);
  io.get(&c->had_init, 4);
  io.get(&c->next_batch, 4);
  io.get(&c->sigma, 4);
  io.get(&T, 8);
  if (!io.ok) return fail(std::string(path) + ": truncated header");
  const bool sane = c->N >= 1 && c->N <= INT32_MAX && c->d >= 1 && c->C >= 1 && c->C <= kMaxC && c->B >= 1 &&
                    c->B <= c->N && c->s > 0.0 && c->s <= 1.0 && c->iters >= 0 && c->next_batch >= 1 &&
                    c->next_batch <= c->B && T >= 0 && T <= (int64_t)c->next_batch * c->iters &&
                    (c->kind == KKM_RBF || c->kind == KKM_LINEAR || c->kind == KKM_RMSD) &&
                    (c->precision == KKM_FP32 || c->precision == KKM_BF16 || c->precision == KKM_FP8) &&
                    (c->sampling == KKM_STRIDE || c->sampling == KKM_BLOCK) &&
                    (c->early_stop == 0 || c->early_stop == 1) && (c->had_init == 0 || c->had_init == 1);
  if (!sane) return fail(std::string(path) + ": inconsistent checkpoint header");
  const int64_t header = 8 + 8 + 8 + 4 + 4 + 8 + 4 + 4 + 4 + 4 + 8 + 4 * 5 + 4 + 8;
  const int64_t body = (int64_t)c->C * 16 + T * 12 + (int64_t)c->next_batch * 8;
  if ((int64_t)len != header + body) return fail(std::string(path) + ": file length disagrees with its header");
  c->M.resize(c->C);
  c->W.resize(c->C);
  c->omega.resize((size_t)T);
  c->changed.resize((size_t)T);
  c->displacement.resize(c->next_batch);
  io.get(c->M.data(), (size_t)c->C * 8);
  io.get(c->W.data(), (size_t)c->C * 8);
  io.get(c->omega.data(), (size_t)T * 8);
  io.get(c->changed.data(), (size_t)T * 4);
  io.get(c->displacement.data(), (size_t)c->next_batch * 8);
  if (!io.ok) return fail(std::string(path) + ": truncated");
  for (int64_t m : c->M)
    if (m < 0 || m >= c->N) return fail(std::string(path) + ": medoid index out of range");
  *out = c.release();
  return KKM_OK;
}

}  // namespace kkm

extern "C" kkm_status kkm_model_save(const kkm_model* m, const char* path) {
  kkm::set_error("");
  try {
    return kkm::save_impl(m, path);
  } catch (...) {
    kkm::set_error("internal exception");
    return KKM_EINTERNAL;
  }
}

extern "C" kkm_status kkm_model_load(const char* path, kkm_model** out) {
  kkm::set_error("");
  try {
    return kkm::load_impl(path, out);
  } catch (...) {
    kkm::set_error("internal exception");
    return KKM_EINTERNAL;
  }
}

extern "C" kkm_status kkm_checkpoint_save(const kkm_checkpoint* c, const char* path) {
  kkm::set_error("");
  try {
    return kkm::ckpt_save_impl(c, path);
  } catch (...) {
    kkm::set_error("internal exception");
    return KKM_EINTERNAL;
  }
}

extern "C" kkm_status kkm_checkpoint_load(const char* path, kkm_checkpoint** out) {
  kkm::set_error("");
  try {
    return kkm::ckpt_load_impl(path, out);
  } catch (...) {
    kkm::set_error("internal exception");
    return KKM_EINTERNAL;
  }
}
