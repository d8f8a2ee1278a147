// Batched frames (lbl_batch_*, include/lbl.h): many frames' transforms and
// labels in a few graph-capturable launches shared by all of them.
#include <algorithm>
#include <new>
#include <vector>

#include "lbl_internal.cuh"

using namespace lbl;

struct lbl_batch_s {
  std::shared_ptr<UseLog> uses = std::make_shared<UseLog>();
  int device = 0;
  int num_sms = 1;
  int32_t n = 0;
  std::vector<lbl_roadmap> rms;
  std::vector<int32_t> P;
  std::vector<lbl_monitor> mons;
  int64_t *part = nullptr;  // every item's partition, concatenated
  unsigned long long *counter = nullptr;  // next work unit of each class's label launch
  int ctas = 1;
  // per class: CTAs per SM of its label launch and work units per warp (set
  // by lbl_batch_create, replaced by lbl_batch_autotune, whose partitions are
  // kept in tuned_parts; partitions they replace stay allocated until
  // lbl_batch_free, so graphs captured before still read live memory)
  int ctas_c[kWordClasses] = {1, 1, 1, 1};
  int upw_c[kWordClasses] = {0, 0, 0, 0};
  std::vector<int64_t *> tuned_parts;
  // items grouped by gathered word width (class c = 1, 2, 4, 8 bytes); item i
  // is entry slot[i] of tabs[cls[i]]
  BatchTable tabs[kWordClasses]{};
  std::vector<int> cls, slot;
  FrameTable ftab{};
  // items whose roadmap has the quadtree form label from their own pyramid
  uint64_t *pyr = nullptr;      // every such item's pyramid, concatenated
  std::vector<int> pyr_slot;    // item -> entry of ptab, or -1
  PyrTable ptab{};
  // frames whose world has at most kPackedWorldRatio times the agent's cells
  // are packed (one launch) and transformed from 64-bit words; the words
  // buffer grows on demand, and a replaced buffer is kept until the batch is
  // freed so graphs captured before still see live memory
  PackTable pktab{};
  uint64_t *words = nullptr;
  int64_t words_cap = 0;
  std::vector<uint64_t *> retired;
  bool frames_set = false;
};

namespace {

// Work units of the batch: the persistent grid's warps take them from a
// counter.  Items are cut into units of about equal cost (nonzeros, or
// quadtree entries, + kEdgeCost per edge), about `upw` per warp overall, at
// least one per item with edges and never more than its edges.
constexpr int64_t kUnitsPerWarp = 8;

int64_t item_cost(const Roadmap &r) { return (r.has_qd ? r.n_qd : r.nnz) + kEdgeCost * r.E; }

// A new plan for the items of class c: partitions in a fresh device buffer
// (*part_out, the caller's to free) and the table's unit ranges rewritten.
cudaError_t plan_class(const lbl_batch_s *b, int c, int ctas, int upw, BatchTable *tab, int64_t **part_out) {
  *part_out = nullptr;
  const int64_t units_target = static_cast<int64_t>(b->num_sms) * ctas * (kThreads / 32) * upw;
  double total = 0.0;
  for (int i = 0; i < b->n; ++i)
    if (b->cls[i] == c) total += static_cast<double>(item_cost(*b->rms[i]));
  const double unit_cost = std::max(total / static_cast<double>(units_target), 1.0);
  std::vector<int64_t> W(b->n, 0), off(b->n + 1, 0);
  for (int i = 0; i < b->n; ++i) {
    const Roadmap &r = *b->rms[i];
    if (b->cls[i] == c && r.E > 0) {
      W[i] = std::max<int64_t>(1, static_cast<int64_t>(std::ceil(static_cast<double>(item_cost(r)) / unit_cost)));
      W[i] = std::min<int64_t>(W[i], r.E);
    }
    off[i + 1] = off[i] + (b->cls[i] == c ? W[i] + 1 : 0);
  }
  int64_t *part = nullptr;
  cudaError_t e = obj_alloc(&part, static_cast<size_t>(std::max<int64_t>(off[b->n], 1)), nullptr);
  if (e != cudaSuccess) return e;
  tab->total = 0;
  for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
    if (b->cls[i] != c) continue;
    const Roadmap &r = *b->rms[i];
    const bool quad = r.has_qd && r.E > 0;
    e = launch_partition_into(quad ? r.qd_rowptr : r.rowptr, r.E, W[i], part + off[i], nullptr);
    BatchItem &it = tab->items[b->slot[i]];
    it.part = part + off[i];
    it.warp0 = tab->total;
    it.warps = W[i];
    tab->total += W[i];
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);  // the partitions, made on the legacy stream
  if (e != cudaSuccess) {
    obj_free_now(part);
    return e;
  }
  *part_out = part;
  return cudaSuccess;
}

}  // namespace

extern "C" {

int lbl_batch_create(int32_t n, const lbl_roadmap *rms, const int32_t *n_props, const lbl_monitor *mons,
                     int32_t ctas_per_sm, lbl_batch *out) {
  clear_error();
  if (!out) {
    set_error("batch create: out is NULL");
    return LBL_EINVAL;
  }
  *out = nullptr;
  if (n < 1 || n > kMaxBatch || !rms || !n_props) {
    set_error("batch create: need 1 <= n <= %d roadmaps and their proposition counts", kMaxBatch);
    return LBL_EINVAL;
  }
  for (int i = 0; i < n; ++i) {
    if (!rms[i] || n_props[i] < 0 || n_props[i] > 64) {
      set_error("batch create: item %d has no roadmap or n_props outside 0..64", i);
      return LBL_EINVAL;
    }
    if (rms[i]->device != rms[0]->device || (mons && mons[i] && mons[i]->device != rms[0]->device)) {
      set_error("batch create: items live on different devices");
      return LBL_EINVAL;
    }
  }
  if (!same_device(rms[0]->device)) return LBL_EINVAL;
  lbl_batch_s *b = new (std::nothrow) lbl_batch_s();
  if (!b) {
    set_error("batch create: out of host memory");
    return LBL_ENOMEM;
  }
  b->device = rms[0]->device;
  b->num_sms = rms[0]->num_sms;
  b->n = n;
  b->rms.assign(rms, rms + n);
  b->P.assign(n_props, n_props + n);
  b->mons.assign(n, nullptr);
  if (mons) b->mons.assign(mons, mons + n);
  // The persistent grid's warps take work units from a counter; items are
  // cut into units of about equal cost (nonzeros + kEdgeCost per edge),
  // kUnitsPerWarp per warp overall, at least one per item with edges.
  bool all_quad = true;
  for (int i = 0; i < n; ++i) all_quad = all_quad && (rms[i]->has_qd || rms[i]->E == 0);
  const int depth = all_quad ? kQuadDepth : 8;
  for (BatchTable &t : b->tabs) t.depth = depth;
  const int occ = batch_ctas_per_sm(depth);
  const int ctas = ctas_per_sm > 0 ? std::min<int>(ctas_per_sm, occ) : occ;
  b->ctas = ctas;
  for (int c = 0; c < kWordClasses; ++c) {
    b->ctas_c[c] = ctas;
    b->upw_c[c] = static_cast<int>(kUnitsPerWarp);
  }
  const int64_t units_target = static_cast<int64_t>(b->num_sms) * ctas * (kThreads / 32) * kUnitsPerWarp;
  // entries streamed per item: quadtree entries when the roadmap has them;
  // word width of its gathers (items of one width share a launch)
  auto entries = [](const Roadmap &r) { return r.has_qd ? r.n_qd : r.nnz; };
  auto width = [&](int i) { return rms[i]->has_qd && rms[i]->E > 0 ? quad_word_bytes(*rms[i], n_props[i]) : 8; };
  // every class's launch gets about kUnitsPerWarp units per warp of its own
  double total[kWordClasses] = {0, 0, 0, 0};
  for (int i = 0; i < n; ++i) total[word_class(width(i))] += static_cast<double>(entries(*rms[i]) + kEdgeCost * rms[i]->E);
  std::vector<int64_t> W(n), off(n + 1, 0);
  int64_t pyr_words = 0;
  for (int i = 0; i < n; ++i)
    if (rms[i]->has_qd && rms[i]->E > 0) pyr_words += rms[i]->pyr_words;
  for (int i = 0; i < n; ++i) {
    const Roadmap &r = *rms[i];
    W[i] = 0;
    if (r.E > 0) {
      const double c = static_cast<double>(entries(r) + kEdgeCost * r.E);
      const double unit_cost = total[word_class(width(i))] / static_cast<double>(units_target);
      W[i] = std::max<int64_t>(1, static_cast<int64_t>(std::ceil(c / unit_cost)));
      W[i] = std::min<int64_t>(W[i], r.E);  // never more units than edges
    }
    off[i + 1] = off[i] + W[i] + 1;
  }
  cudaError_t e = obj_alloc(&b->part, static_cast<size_t>(off[n]), nullptr);
  if (e == cudaSuccess) e = obj_alloc(&b->counter, kWordClasses, nullptr);
  if (e == cudaSuccess && pyr_words > 0) e = obj_alloc(&b->pyr, static_cast<size_t>(pyr_words), nullptr);
  b->pyr_slot.assign(n, -1);
  b->cls.assign(n, kWordClasses - 1);
  b->slot.assign(n, 0);
  int64_t pyr0 = 0, block0 = 0;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const Roadmap &r = *rms[i];
    const bool quad = r.has_qd && r.E > 0;
    const int wb = width(i);
    e = launch_partition_into(quad ? r.qd_rowptr : r.rowptr, r.E, W[i], b->part + off[i], nullptr);
    BatchTable &tb = b->tabs[word_class(wb)];
    b->cls[i] = word_class(wb);
    b->slot[i] = tb.n;
    tb.word_bytes = wb;
    BatchItem &it = tb.items[tb.n++];
    it = BatchItem{};
    it.rowptr = quad ? r.qd_rowptr : r.rowptr;
    it.colidx = quad ? r.qd_idx : r.colidx;
    it.perm = quad ? r.qd_perm : nullptr;
    it.part = b->part + off[i];
    if (quad) {  // labels gather from the item's pyramid, built from its O at the label stage
      PyrItem &pi = b->ptab.items[b->ptab.n];
      pi = PyrItem{};
      pi.pyr = b->pyr + pyr0;
      pi.cells = r.cells;
      pi.block0 = block0;
      pi.off = r.qd_off;
      pi.word_bytes = wb;
      pi.tiled_w = r.qd_tiled_w;
      it.O = pi.pyr;
      b->pyr_slot[i] = b->ptab.n++;
      pyr0 += r.pyr_words;
      block0 += (r.cells + kThreads - 1) / kThreads;
    }
    it.mask = n_props[i] >= 64 ? ~0ull : ((1ull << n_props[i]) - 1ull);
    it.warp0 = tb.total;  // work units of this class's launch
    it.warps = W[i];
    if (b->mons[i]) {
      const Monitor &m = *b->mons[i];
      it.T = m.T;
      it.V = m.V;
      it.m = m.m;
      for (int j = 0; j < 8; ++j) it.rel[j] = m.rel[j];
    }
    tb.total += W[i];
    if (entries(r) >= kNarrowLimit || r.E >= kNarrowLimit) tb.wide = 1;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  if (e != cudaSuccess) {
    b->uses->release(b->device, {b->part, b->counter, b->pyr});
    delete b;
    return cuda_fail(e, "batch create: partitions");
  }
  b->ptab.total = block0;
  b->ftab.n = n;
  *out = b;
  return LBL_OK;
}

int lbl_batch_set_frames(lbl_batch b, const lbl_frame *frames) {
  clear_error();
  if (!b || !frames) {
    set_error("batch frames: NULL batch or frames");
    return LBL_EINVAL;
  }
  int64_t cell0 = 0;
  for (int i = 0; i < b->n; ++i) {
    const lbl_frame &f = frames[i];
    const Roadmap &r = *b->rms[i];
    const int32_t P = b->P[i];
    if (!valid_grid(&f.world, "batch frames (world)", false)) return LBL_EINVAL;
    if ((P > 0 && !f.d_planes) || !f.d_O || (r.E > 0 && !f.d_L) ||
        (b->mons[i] && r.E > 0 && (!f.d_next || !f.d_viol))) {
      set_error("batch frames: frame %d is missing a buffer", i);
      return LBL_EINVAL;
    }
    FrameMap m;
    if (!frame_map(f.world, r.agent, f.pose, &m)) return LBL_EINVAL;
    b->ftab.items[i] = frame_item(m, f.world, r.agent, f.d_planes, P, f.d_O, cell0);
    cell0 += r.cells;
    BatchItem &it = b->tabs[b->cls[i]].items[b->slot[i]];
    if (b->pyr_slot[i] >= 0)
      b->ptab.items[b->pyr_slot[i]].O = f.d_O;  // the item gathers from its pyramid
    else
      it.O = f.d_O;
    it.L = f.d_L;
    it.next = f.d_next;
    it.viol = f.d_viol;
  }
  b->ftab.total = cell0;
  // packed frames: 64-bit words at 4-word aligned offsets (vector stores)
  int64_t need = 0;
  std::vector<int64_t> woff(b->n, -1);
  for (int i = 0; i < b->n; ++i) {
    const int64_t wc = grid_cells(frames[i].world);
    if (b->P[i] > 0 && wc > 0 && wc <= kPackedWorldRatio * b->rms[i]->cells) {
      woff[i] = need;
      need += (wc + 3) / 4 * 4;
    }
  }
  if (need > b->words_cap) {
    uint64_t *w = nullptr;
    cudaError_t e = obj_alloc(&w, static_cast<size_t>(need), nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "batch frames: packed words");
    if (b->words) b->retired.push_back(b->words);
    b->words = w;
    b->words_cap = need;
  }
  PackTable &pt = b->pktab;
  pt.n = 0;
  pt.lane0[0] = 0;
  for (int i = 0; i < b->n; ++i) {
    FrameItem &fi = b->ftab.items[i];
    fi.words = nullptr;
    if (woff[i] < 0) continue;
    const int32_t P = b->P[i];
    const PackItem it{frames[i].d_planes, b->words + woff[i], grid_cells(frames[i].world), P, 8};
    pt.items[pt.n] = it;
    pt.vec[pt.n] = pack_vec_ok(it) ? 1 : 0;
    pt.lane0[pt.n + 1] = pt.lane0[pt.n] + (it.cells + 3) / 4;
    ++pt.n;
    fi.words = it.words;
    fi.word_bytes = 8;
    fi.wmask = P >= 64 ? ~0ull : ((1ull << P) - 1ull);
  }
  b->frames_set = true;
  return LBL_OK;
}

int lbl_batch_launch(lbl_batch b, uint32_t stages, lbl_stream s) {
  clear_error();
  if (!b || !b->frames_set || (stages & ~(LBL_STAGE_TRANSFORM | LBL_STAGE_LABEL))) {
    set_error("batch launch: NULL batch, no frames set, or unknown stages");
    return LBL_EINVAL;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  cudaError_t e = cudaSuccess;
  if (stages & LBL_STAGE_TRANSFORM) {
    e = launch_pack_batch(b->pktab, st);
    if (e == cudaSuccess) e = launch_frame_batch(b->ftab, b->num_sms, st);
  }
  if (e == cudaSuccess && (stages & LBL_STAGE_LABEL)) {
    e = launch_quad_pyramid_batch(b->ptab, st);
    for (int c = 0; c < kWordClasses && e == cudaSuccess; ++c)
      if (b->tabs[c].n > 0) e = launch_label_batch(b->tabs[c], b->counter + c, b->num_sms, b->ctas_c[c], st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  // the batch's memory, and its roadmaps' rows and monitors' tables, are in use
  // until this launch ends (not logged while the stream is being captured)
  b->uses->note(st);
  for (int i = 0; i < b->n; ++i) {
    if (i == 0 || b->rms[i] != b->rms[i - 1]) b->rms[i]->uses->note(st);
    if (b->mons[i]) b->mons[i]->uses->note(st);
  }
  return LBL_OK;
}

int lbl_batch_free(lbl_batch b) {
  clear_error();
  if (!b) return LBL_OK;
  // released after the batch's last logged launch, without waiting for the device
  std::vector<void *> mem = {b->part, b->counter, b->pyr, b->words};
  for (uint64_t *w : b->retired) mem.push_back(w);
  for (int64_t *q : b->tuned_parts) mem.push_back(q);
  b->uses->release(b->device, mem);
  delete b;
  return LBL_OK;
}

int lbl_batch_autotune(lbl_batch b, int32_t reps, lbl_stream s, lbl_batch_tuning *out) {
  clear_error();
  if (!b || !b->frames_set || reps < 1 || reps > 1000) {
    set_error("batch autotune: NULL batch, no frames set, or reps outside 1..1000");
    return LBL_EINVAL;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  // the frames' agent words and pyramids, which every candidate reads
  int rc = lbl_batch_launch(b, LBL_STAGE_TRANSFORM | LBL_STAGE_LABEL, s);
  if (rc != LBL_OK) return rc;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  // mean time of `reps` launches of one class's labels under a candidate plan
  auto time_class = [&](int c, const BatchTable &tab, int ctas, float *ms) {
    cudaError_t r = launch_label_batch(tab, b->counter + c, b->num_sms, ctas, st);  // untimed
    if (r == cudaSuccess) r = cudaEventRecord(t0, st);
    for (int i = 0; i < reps && r == cudaSuccess; ++i) r = launch_label_batch(tab, b->counter + c, b->num_sms, ctas, st);
    if (r == cudaSuccess) r = cudaEventRecord(t1, st);
    if (r == cudaSuccess) r = cudaEventSynchronize(t1);
    if (r == cudaSuccess) r = cudaEventElapsedTime(ms, t0, t1);
    *ms /= static_cast<float>(reps);
    return r;
  };
  for (int c = 0; c < kWordClasses && e == cudaSuccess; ++c) {
    lbl_batch_tuning res{};
    BatchTable &cur = b->tabs[c];
    if (cur.n == 0) {
      if (out) out[c] = res;
      continue;
    }
    res.word_bytes = cur.word_bytes ? cur.word_bytes : 8;
    res.items = cur.n;
    float best_ms = 0.0f;
    e = time_class(c, cur, b->ctas_c[c], &best_ms);
    res.ms_default = best_ms;
    int best_depth = cur.depth, best_ctas = b->ctas_c[c], best_upw = b->upw_c[c];
    int64_t *best_part = nullptr;
    BatchTable best_tab = cur;
    // candidates: register depth, CTAs per SM (up to what fits), work units per warp
    for (int depth : {8, 12}) {
      if (depth == 12 && cur.wide) continue;  // the 64-bit range kernel exists at depth 8 only
      const int occ = batch_ctas_per_sm(depth);
      for (int ctas = occ; ctas >= std::max(1, occ - 2) && e == cudaSuccess; --ctas) {
        for (int upw : {2, 4, 8, 16, 32}) {
          BatchTable tab = cur;
          tab.depth = depth;
          int64_t *part = nullptr;
          e = plan_class(b, c, ctas, upw, &tab, &part);
          float ms = 0.0f;
          if (e == cudaSuccess) e = time_class(c, tab, ctas, &ms);
          if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best_depth = depth;
            best_ctas = ctas;
            best_upw = upw;
            best_tab = tab;
            std::swap(best_part, part);
          }
          obj_free_now(part);  // its timed launches have completed
          if (e != cudaSuccess) break;
        }
      }
    }
    if (e == cudaSuccess && best_part) {  // adopt the winner; the plan it replaces stays allocated
      cur = best_tab;
      b->ctas_c[c] = best_ctas;
      b->upw_c[c] = best_upw;
      b->tuned_parts.push_back(best_part);
      best_part = nullptr;
    }
    obj_free_now(best_part);
    res.depth = best_depth;
    res.ctas_per_sm = best_ctas;
    res.units_per_warp = best_upw;
    res.ms = best_ms;
    if (out) out[c] = res;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (e != cudaSuccess) return cuda_fail(e, "batch autotune");
  return LBL_OK;
}

}  // extern "C"
