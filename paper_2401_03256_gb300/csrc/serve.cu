// serve.cu - serving form: a request loop over several resident graphs.
//
// Every attached graph has a FIFO of update requests and one worker thread, so each graph
// has a single writer and its requests run in arrival order (Section 3.2: one writer on
// the graph at a time).  A request is admitted when one of `slots` device slots is free
// and cudaMemGetInfo shows at least `hbm_reserve_bytes` plus the request's estimate free;
// admitted requests of different graphs run at the same time on their graphs' own
// streams.  Each graph's persistent rank launch is sized to 1/slots of the blocks that can
// be resident, so the cooperative kernels of concurrent requests always fit on the device
// together.  Continuous batching: when a graph's worker gets a slot it takes the requests
// queued for that graph by then (up to max_coalesce), applies their batches in order with
// one pr_apply_batches and runs one pr_dynamic_frontier over the net change;
// each result records submit, start and completion times (host clock) and the stats.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "prdf_graph.cuh"


namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket;
  int32_t graph;
  std::vector<uint32_t> del_src, del_dst, ins_src, ins_dst;
  double t_submit;
};

}  // namespace

struct pr_server {
  pr_server_config cfg{};
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_slot;
  std::vector<pr_graph *> graphs;
  std::vector<std::deque<Request>> queues;
  std::vector<std::thread> workers;
  std::map<uint64_t, pr_request_result> done;
  uint64_t next_ticket = 1;
  int32_t busy_slots = 0;
  uint64_t admitted = 0, waited_for_memory = 0;
  int64_t pending = 0;
  bool stopping = false;

  double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

namespace {

// Device memory a request may allocate: batch scratch (about 128 bytes per pair) plus room
// for moved rows and a repack of the larger adjacency's column array.
uint64_t request_estimate(const pr_graph *h, uint64_t pairs) {
  const prdf::Graph &g = h->g;
  uint64_t cols = std::max(g.out.col_cap, g.in.col_cap) * 4ull;
  return 128ull * pairs + cols / 8 + (16ull << 20);
}

// The group's batches concatenated in submission order, applied by one pr_apply_batches.
pr_status apply_group(pr_graph *h, const std::vector<Request> &group) {
  const size_t nb = group.size();
  std::vector<int64_t> doff(nb + 1, 0), ioff(nb + 1, 0);
  for (size_t k = 0; k < nb; k++) {
    doff[k + 1] = doff[k] + (int64_t)group[k].del_src.size();
    ioff[k + 1] = ioff[k] + (int64_t)group[k].ins_src.size();
  }
  std::vector<uint32_t> ds, dd, is, id;
  ds.reserve(doff[nb]);
  dd.reserve(doff[nb]);
  is.reserve(ioff[nb]);
  id.reserve(ioff[nb]);
  for (const Request &rq : group) {
    ds.insert(ds.end(), rq.del_src.begin(), rq.del_src.end());
    dd.insert(dd.end(), rq.del_dst.begin(), rq.del_dst.end());
    is.insert(is.end(), rq.ins_src.begin(), rq.ins_src.end());
    id.insert(id.end(), rq.ins_dst.begin(), rq.ins_dst.end());
  }
  return pr_apply_batches(h, (int32_t)nb, doff.data(), ds.data(), dd.data(), ioff.data(), is.data(), id.data());
}

void worker_loop(pr_server *s, int32_t gi) {
  pr_graph *h = s->graphs[gi];
  for (;;) {
    std::vector<Request> group;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stopping || !s->queues[gi].empty(); });
      if (s->queues[gi].empty()) return;  // stopping and drained
      // admission: a free slot and enough free device memory for the head request
      const Request &head = s->queues[gi].front();
      const uint64_t need = request_estimate(h, head.del_src.size() + head.ins_src.size()) + s->cfg.hbm_reserve_bytes;
      bool counted = false;
      for (;;) {
        if (s->busy_slots < s->cfg.slots) {
          size_t free_b = 0, total_b = 0;
          int dev = -1;
          cudaGetDevice(&dev);
          if (dev != h->g.device) cudaSetDevice(h->g.device);
          if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            free_b = 0;
          }
          if (free_b >= need || s->busy_slots == 0) break;  // an idle device always admits one
          if (!counted) {
            s->waited_for_memory++;
            counted = true;
          }
        }
        s->cv_slot.wait_for(lk, std::chrono::milliseconds(1));
      }
      s->busy_slots++;
      s->admitted++;
      // continuous batching: the requests of this graph queued by now are served together
      while (!s->queues[gi].empty() && (int32_t)group.size() < s->cfg.max_coalesce) {
        group.push_back(std::move(s->queues[gi].front()));
        s->queues[gi].pop_front();
      }
    }
    const double t_start = s->now_ms();
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != h->g.device) cudaSetDevice(h->g.device);
    std::vector<pr_status> st(group.size(), PR_OK);
    bool any = false;
    if (group.size() == 1) {
      const Request &rq = group[0];
      st[0] = pr_apply_batch(h, (int64_t)rq.del_src.size(), rq.del_src.data(), rq.del_dst.data(),
                             (int64_t)rq.ins_src.size(), rq.ins_src.data(), rq.ins_dst.data());
      any = st[0] == PR_OK;
    } else {
      // one sequence apply for the whole group; if it is rejected (the graph is then
      // unchanged), each request is applied alone so that only the bad ones fail
      pr_status all = apply_group(h, group);
      if (all == PR_OK) {
        any = true;
      } else if (all == PR_ERR_VERTEX_RANGE || all == PR_ERR_INVALID_ARG) {
        for (size_t k = 0; k < group.size(); k++) {
          const Request &rq = group[k];
          st[k] = pr_apply_batch(h, (int64_t)rq.del_src.size(), rq.del_src.data(), rq.del_dst.data(),
                                 (int64_t)rq.ins_src.size(), rq.ins_src.data(), rq.ins_dst.data());
          any = any || st[k] == PR_OK;
        }
      } else {
        std::fill(st.begin(), st.end(), all);
      }
    }
    pr_stats stats{};
    pr_status df = any ? pr_dynamic_frontier(h, &stats) : PR_OK;
    const double t_done = s->now_ms();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (size_t k = 0; k < group.size(); k++) {
        pr_request_result r{};
        r.ticket = group[k].ticket;
        r.graph = gi;
        r.status = st[k] != PR_OK ? st[k] : df;
        r.t_submit_ms = group[k].t_submit;
        r.t_start_ms = t_start;
        r.t_done_ms = t_done;
        r.coalesced = (int32_t)group.size();
        r.stats = stats;
        s->done[r.ticket] = r;
      }
      s->busy_slots--;
      s->pending -= (int64_t)group.size();
    }
    s->cv_slot.notify_all();
    s->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

void pr_server_config_default(pr_server_config *c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->slots = 2;
  c->max_coalesce = 256;
  c->hbm_reserve_bytes = 1ull << 30;
}

pr_status pr_server_create(const pr_server_config *cfg, pr_server **out) {
  if (!out) return PR_ERR_INVALID_ARG;
  *out = nullptr;
  pr_server_config c;
  if (cfg) c = *cfg; else pr_server_config_default(&c);
  if (c.slots < 1 || c.slots > 64 || c.max_coalesce < 1 || c.max_coalesce > PR_MAX_BATCHES) return PR_ERR_INVALID_ARG;
  pr_server *s = new (std::nothrow) pr_server;
  if (!s) return PR_ERR_OUT_OF_MEMORY;
  s->cfg = c;
  s->t0 = Clock::now();
  *out = s;
  return PR_OK;
}

pr_status pr_server_add_graph(pr_server *s, pr_graph *g, int32_t *index) {
  if (!s || !g) return PR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping || s->graphs.size() >= 1024) return PR_ERR_INVALID_ARG;
  // 1/slots of the resident blocks, so concurrent requests' cooperative launches fit together
  g->g.rank_grid = std::max(1, g->g.rank_grid_max / s->cfg.slots);
  int32_t gi = (int32_t)s->graphs.size();
  s->graphs.push_back(g);
  s->queues.emplace_back();
  s->workers.emplace_back(worker_loop, s, gi);
  if (index) *index = gi;
  return PR_OK;
}

pr_status pr_server_submit(pr_server *s, int32_t graph, int64_t n_del, const uint32_t *del_src,
                           const uint32_t *del_dst, int64_t n_ins, const uint32_t *ins_src, const uint32_t *ins_dst,
                           uint64_t *ticket) {
  if (!s || !ticket || n_del < 0 || n_ins < 0) return PR_ERR_INVALID_ARG;
  if ((n_del && (!del_src || !del_dst)) || (n_ins && (!ins_src || !ins_dst))) return PR_ERR_INVALID_ARG;
  Request rq;
  rq.del_src.assign(del_src, del_src + n_del);
  rq.del_dst.assign(del_dst, del_dst + n_del);
  rq.ins_src.assign(ins_src, ins_src + n_ins);
  rq.ins_dst.assign(ins_dst, ins_dst + n_ins);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping || graph < 0 || graph >= (int32_t)s->graphs.size()) return PR_ERR_INVALID_ARG;
    rq.ticket = s->next_ticket++;
    rq.graph = graph;
    rq.t_submit = s->now_ms();
    *ticket = rq.ticket;
    s->queues[graph].push_back(std::move(rq));
    s->pending++;
  }
  s->cv_work.notify_all();
  return PR_OK;
}

pr_status pr_server_wait(pr_server *s, uint64_t ticket, pr_request_result *out) {
  if (!s) return PR_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (ticket == 0 || ticket >= s->next_ticket) return PR_ERR_INVALID_ARG;
  s->cv_done.wait(lk, [&] { return s->done.count(ticket) != 0; });
  if (out) *out = s->done[ticket];
  return PR_OK;
}

pr_status pr_server_drain(pr_server *s, pr_server_info *info) {
  if (!s) return PR_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [&] { return s->pending == 0; });
  if (info) {
    info->submitted = (int64_t)(s->next_ticket - 1);
    info->completed = (int64_t)s->done.size();
    info->waited_for_memory = (int64_t)s->waited_for_memory;
    info->elapsed_ms = s->now_ms();
  }
  return PR_OK;
}

pr_status pr_server_destroy(pr_server *s) {
  if (!s) return PR_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->workers) t.join();
  delete s;
  return PR_OK;
}

}  // extern "C"
