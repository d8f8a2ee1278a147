// Host-buffer frames (lbl_session_*, include/lbl.h): planes in, transform,
// labels and monitor outputs out, with copies overlapping the kernels.
#include <algorithm>
#include <new>
#include <vector>

#include "lbl_internal.cuh"

using namespace lbl;

struct lbl_session_s {
  std::shared_ptr<UseLog> uses = std::make_shared<UseLog>();  // the caller's streams the session's work waited on
  int device = 0;
  lbl_roadmap rm = nullptr;
  lbl_monitor mon = nullptr;
  lbl_grid world{};
  int32_t P = 0;
  lbl_config cfg{};
  bool has_cfg = false;
  uint8_t *planes = nullptr;
  uint64_t *O = nullptr, *L = nullptr, *next = nullptr;
  uint16_t *viol = nullptr;
  // Two plane buffers, filled on `cin` in turn: frame i+1's planes go to the
  // device while frame i is transformed and labeled.  ev_in[k]: slot k filled;
  // ev_free[k]: the frame that read slot k is done (recorded after its labels,
  // so no event separates the frame's kernels).
  uint8_t *slot[2] = {nullptr, nullptr};
  cudaStream_t cin = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  int64_t frame = 0;
  // The session's kernels run on `cc`, and its outputs go to one of two device
  // buffer sets in turn, so frame i+1 computes while frame i's results are
  // still being copied out; ev_out[k]: output set k copied to the host.
  cudaStream_t cc = nullptr;
  uint64_t *Ls[2] = {nullptr, nullptr}, *Ns[2] = {nullptr, nullptr};
  uint16_t *Vs[2] = {nullptr, nullptr};
  cudaEvent_t ev_out[2] = {nullptr, nullptr};
  uint64_t *pyr = nullptr;  // the session's own quadtree pyramid (chunked quadtree sessions)
  // Packed world words: the planes are packed (one coalesced pass) and the
  // transform gathers one word per agent cell.  Used for planes of at least
  // kPackedMinPlaneBytes on a world of at most kPackedWorldRatio times the
  // agent's cells, so packing reads little the transform would not.
  uint8_t *words = nullptr;
  // Own-stream labeling (`chunked`, with the default form: quadtree, else
  // streaming CSR, on roadmaps of kSessionChunkMinEdges edges or more): the
  // session's own pyramid and partition, its kernels on `cc`, the results
  // copied to the host on `cs`.  The whole roadmap is one range, labeled by the
  // moving front or the per-warp stream as lbl_label chooses by size; frames
  // run back to back overlap one frame's copies with the next frame's kernels
  // through the two output sets.  (Four ranges, each copied out while the next
  // was labeled, measured slower at every size: 100k edges 0.055 vs 0.036 ms
  // per frame, 250k 0.117 vs 0.089, 400k 0.155 vs 0.129, 1M 0.29 vs 0.26.)
  bool chunked = false;
  bool quad = false;
  int depth = 8, ctas = 0;
  int64_t *cpart = nullptr;  // the warps' partition: warps + 1 entries
  int64_t warps = 0;
  int front_chunk = -1;  // quadtree: -1 = the moving front by size (as lbl_label), 0 = per-warp stream, > 0 = front
  cudaStream_t cs = nullptr;
  cudaEvent_t ev = nullptr;  // labels done: the copies on `cs` may start
};

extern "C" {

int lbl_session_create(lbl_roadmap rm, const lbl_grid *world, int32_t n_props, lbl_monitor mon,
                       const lbl_config *cfg, lbl_session *out) {
  clear_error();
  if (!out) {
    set_error("session create: out is NULL");
    return LBL_EINVAL;
  }
  *out = nullptr;
  if (!rm) {
    set_error("session create: NULL roadmap");
    return LBL_EINVAL;
  }
  if (!valid_grid(world, "session create (world)", false)) return LBL_EINVAL;
  if (n_props < 0 || n_props > 64) {
    set_error("session create: n_props = %d outside 0..64", n_props);
    return LBL_EINVAL;
  }
  if (!same_device(rm->device)) return LBL_EINVAL;
  lbl_session_s *ss = new (std::nothrow) lbl_session_s();
  if (!ss) {
    set_error("session create: out of host memory");
    return LBL_ENOMEM;
  }
  ss->device = rm->device;
  ss->rm = rm;
  ss->mon = mon;
  ss->world = *world;
  ss->P = n_props;
  if (cfg) {
    ss->cfg = *cfg;
    ss->has_cfg = true;
  }
  const size_t plane_bytes = static_cast<size_t>(n_props) * grid_cells(*world);
  cudaError_t e = obj_alloc(&ss->planes, 2 * plane_bytes, nullptr);
  ss->slot[0] = ss->planes;
  ss->slot[1] = ss->planes + plane_bytes;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ss->cin, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&ss->ev_in[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ss->ev_free[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = obj_alloc(&ss->O, static_cast<size_t>(rm->cells), nullptr);
  if (e == cudaSuccess && static_cast<int64_t>(plane_bytes) >= kPackedMinPlaneBytes &&
      grid_cells(*world) <= kPackedWorldRatio * rm->cells)
    e = obj_alloc(&ss->words, static_cast<size_t>(grid_cells(*world)) * packed_word_bytes(n_props), nullptr);
  if (e == cudaSuccess) e = obj_alloc(&ss->L, static_cast<size_t>(2 * rm->E), nullptr);
  if (e == cudaSuccess && mon) e = obj_alloc(&ss->next, static_cast<size_t>(2 * rm->E), nullptr);
  if (e == cudaSuccess && mon) e = obj_alloc(&ss->viol, static_cast<size_t>(2 * rm->E), nullptr);
  for (int k = 0; k < 2; ++k) {
    ss->Ls[k] = ss->L ? ss->L + k * rm->E : nullptr;
    ss->Ns[k] = ss->next ? ss->next + k * rm->E : nullptr;
    ss->Vs[k] = ss->viol ? ss->viol + k * rm->E : nullptr;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ss->cc, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ss->ev_out[k], cudaEventDisableTiming);

  // Own-stream labeling when the configuration resolves to a register-pipelined
  // stream (quadtree, or CSR without lane groups, early exit or copy rings) on
  // a roadmap big enough to pay.
  lbl_config c{};
  if (cfg) c = *cfg;
  if (c.algo == LBL_ALGO_AUTO && rm->tuned_valid[n_props]) c = rm->tuned[n_props];
  if (c.algo == LBL_ALGO_AUTO)  // as lbl_label resolves it
    c.algo = rm->has_qd ? LBL_ALGO_QUAD : (rm->has_bt && n_props <= 8) ? LBL_ALGO_BITTILE : LBL_ALGO_CSR;
  const bool stream_form = (c.algo == LBL_ALGO_QUAD && rm->has_qd) ||
                           (c.algo == LBL_ALGO_CSR && c.lanes_per_edge == 0 && c.early_exit <= 0 &&
                            (c.pipeline == 0 || c.pipeline == LBL_PIPE_REGISTERS));
  if (e == cudaSuccess && stream_form && rm->E >= kSessionChunkMinEdges) {
    ss->chunked = true;
    ss->quad = c.algo == LBL_ALGO_QUAD;
    if (ss->quad) e = obj_alloc(&ss->pyr, static_cast<size_t>(rm->pyr_words), nullptr);
    // quadtree sessions on z-order (or tiled row-major) grids always pack the
    // planes: the transform then builds the pyramid itself (device step 0.0393 -> 0.0376 ms on the
    // 100k-edge frame with 2 MiB of planes)
    if (e == cudaSuccess && ss->quad && !ss->words && n_props > 0 &&
        (rm->agent.order == LBL_ORDER_MORTON || rm->qd_tiled_w > 0) &&
        grid_cells(*world) <= kPackedWorldRatio * rm->cells)
      e = obj_alloc(&ss->words, static_cast<size_t>(grid_cells(*world)) * packed_word_bytes(n_props), nullptr);
    ss->depth = c.depth ? c.depth : (ss->quad ? kQuadDepth : 8);
    const int occ = stream_ctas_per_sm(ss->depth);
    ss->ctas = c.ctas_per_sm > 0 ? std::min(c.ctas_per_sm, occ) : occ;
    ss->warps = static_cast<int64_t>(rm->num_sms) * ss->ctas * (kThreads / 32);
    if (ss->quad && c.pipeline == LBL_PIPE_FRONT) ss->front_chunk = std::max(front_chunk_for(rm->E, rm->num_sms), 8);
    if (!ss->quad || c.pipeline == LBL_PIPE_REGISTERS) ss->front_chunk = 0;
    const int64_t *rows = ss->quad ? rm->qd_rowptr : rm->rowptr;
    e = obj_alloc(&ss->cpart, static_cast<size_t>(ss->warps + 1), nullptr);
    if (e == cudaSuccess) e = launch_partition_into(rows, rm->E, ss->warps, ss->cpart, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ss->cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ss->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    lbl_session_free(ss);
    return cuda_fail(e, "session create");
  }
  *out = ss;
  return LBL_OK;
}

int lbl_session_run(lbl_session ss, const uint8_t *h_planes, lbl_pose pose, uint64_t *h_L, uint64_t *h_next,
                    uint16_t *h_viol, lbl_stream s) {
  clear_error();
  if (!ss) {
    set_error("session run: NULL session");
    return LBL_EINVAL;
  }
  const Roadmap &rm = *ss->rm;
  if ((ss->P > 0 && !h_planes) || (rm.E > 0 && !h_L)) {
    set_error("session run: NULL host buffer");
    return LBL_EINVAL;
  }
  if (!same_device(ss->device)) return LBL_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  // A chunked session touches only its own device memory (planes, O,
  // pyramid, partitions, outputs) besides the roadmap's read-only rows, so
  // its kernels run on its own stream `cc` and frame i+1 computes while frame
  // i's results are still being copied out.  Other sessions label through
  // lbl_label (roadmap-owned working memory), ordered on the caller's stream.
  cudaStream_t cc = ss->chunked ? ss->cc : st;
  const size_t plane_bytes = static_cast<size_t>(ss->P) * grid_cells(ss->world);
  const int k = static_cast<int>(ss->frame & 1);  // plane slot and output set of this frame
  uint64_t *dL = ss->Ls[k], *dN = ss->Ns[k];
  uint16_t *dV = ss->Vs[k];
  // planes in on `cin` once slot k is no longer read
  cudaError_t e = cudaStreamWaitEvent(ss->cin, ss->ev_free[k], 0);
  if (e == cudaSuccess && plane_bytes)
    e = cudaMemcpyAsync(ss->slot[k], h_planes, plane_bytes, cudaMemcpyHostToDevice, ss->cin);
  if (e == cudaSuccess) e = cudaEventRecord(ss->ev_in[k], ss->cin);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cc, ss->ev_in[k], 0);
  // output set k copied out (frame i-2) before this frame's kernels, so no
  // event sits between them and each is launched while the one before ends
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cc, ss->ev_out[k], 0);
  if (e != cudaSuccess) return cuda_fail(e, "session run: copy planes");
  int rc = LBL_OK;
  // quadtree sessions on z-order (or tiled row-major) grids build the pyramid
  // inside the transform (the words are needed only as its level 0, so O is
  // not written)
  const bool fused = ss->words && ss->chunked && ss->quad && (rm.agent.order == LBL_ORDER_MORTON || rm.qd_tiled_w > 0);
  if (ss->words) {
    const PackItem it{ss->slot[k], ss->words, grid_cells(ss->world), ss->P, packed_word_bytes(ss->P)};
    if ((e = launch_pack_planes(it, cc)) != cudaSuccess) return cuda_fail(e, "session run: pack planes");
    if (fused)
      rc = transform_pyramid(&ss->world, ss->words, ss->P, pose, rm, nullptr, ss->pyr, cc);
    else
      rc = lbl_frame_transform_words(&ss->world, ss->words, ss->P, pose, &rm.agent, ss->O,
                                     reinterpret_cast<lbl_stream>(cc));
  } else {
    rc = lbl_frame_transform(&ss->world, ss->slot[k], ss->P, pose, &rm.agent, ss->O, reinterpret_cast<lbl_stream>(cc));
  }
  if (rc != LBL_OK) return rc;
  ++ss->frame;
  auto copy_out = [&](int64_t e0, int64_t n) {
    cudaError_t r = cudaMemcpyAsync(h_L + e0, dL + e0, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, ss->cs);
    if (r == cudaSuccess && ss->mon && h_next)
      r = cudaMemcpyAsync(h_next + e0, dN + e0, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, ss->cs);
    if (r == cudaSuccess && ss->mon && h_viol)
      r = cudaMemcpyAsync(h_viol + e0, dV + e0, sizeof(uint16_t) * n, cudaMemcpyDeviceToHost, ss->cs);
    return r;
  };
  if (ss->chunked) {
    const void *base = ss->O;
    int wb = 8;
    if (ss->quad) {
      wb = quad_word_bytes(rm, ss->P);
      if (!fused && (e = launch_quad_pyramid(rm, ss->O, wb, ss->pyr, cc)) != cudaSuccess)
        return cuda_fail(e, "session run: pyramid");
      base = ss->pyr;
    }
    StreamRows r{ss->quad ? rm.qd_rowptr : rm.rowptr, ss->quad ? rm.qd_idx : rm.colidx, ss->cpart, ss->ctas, rm.E,
                 ss->quad ? rm.n_qd : rm.nnz, ss->quad ? rm.qd_perm : nullptr};
    r.front_chunk = ss->front_chunk;
    MonitorTables t{};
    if (ss->mon) t = tables_of(*ss->mon, dN, dV);
    e = launch_label_rows(r, base, wb, ss->P, dL, ss->mon ? &t : nullptr, ss->depth, rm.num_sms, cc);
    if (e == cudaSuccess) e = cudaEventRecord(ss->ev_free[k], cc);  // plane slot k free (read before the labels)
    if (e == cudaSuccess) e = cudaEventRecord(ss->ev, cc);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ss->cs, ss->ev, 0);
    if (e == cudaSuccess) e = copy_out(0, rm.E);
    if (e != cudaSuccess) return cuda_fail(e, "session run: labels");
  } else {
    rc = label_impl(ss->rm, ss->O, ss->P, dL, ss->mon, dN, dV, ss->has_cfg ? &ss->cfg : nullptr, cc);
    if (rc != LBL_OK) return rc;
    if ((e = cudaEventRecord(ss->ev_free[k], cc)) != cudaSuccess || (e = cudaEventRecord(ss->ev, cc)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(ss->cs, ss->ev, 0)) != cudaSuccess ||
        (rm.E > 0 && (e = copy_out(0, rm.E)) != cudaSuccess))
      return cuda_fail(e, "session run: copy results");
  }
  // output set k is free again once its copies land; the caller's stream sees
  // the whole frame (copies in, kernels, copies out) before its next work
  if ((e = cudaEventRecord(ss->ev_out[k], ss->cs)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(st, ss->ev_out[k], 0)) != cudaSuccess)
    return cuda_fail(e, "session run: join");
  rm.uses->note(cc);  // the roadmap's and monitor's rows and tables were read on the session's streams
  if (ss->mon) ss->mon->uses->note(cc);
  ss->uses->note(st);
  return LBL_OK;
}

int lbl_session_free(lbl_session ss) {
  clear_error();
  if (!ss) return LBL_OK;
  // the session's own streams hold all its work (with the caller's streams it
  // waited on, logged by lbl_session_run): its memory is released after that,
  // without waiting for the rest of the device
  for (cudaStream_t q : {ss->cin, ss->cc, ss->cs})
    if (q) ss->uses->note(q);
  ss->uses->release(ss->device, {ss->planes, ss->O, ss->L, ss->next, ss->viol, ss->cpart, ss->pyr, ss->words});
  if (ss->cs) cudaStreamDestroy(ss->cs);  // destroyed once their work is done
  if (ss->cin) cudaStreamDestroy(ss->cin);
  if (ss->cc) cudaStreamDestroy(ss->cc);
  for (int k = 0; k < 2; ++k)
    if (ss->ev_out[k]) cudaEventDestroy(ss->ev_out[k]);
  if (ss->ev) cudaEventDestroy(ss->ev);
  for (int k = 0; k < 2; ++k) {
    if (ss->ev_in[k]) cudaEventDestroy(ss->ev_in[k]);
    if (ss->ev_free[k]) cudaEventDestroy(ss->ev_free[k]);
  }
  delete ss;
  return LBL_OK;
}

}  // extern "C"
