// Solve server (continuous batching); see serve.cu.
#pragma once
#include <string>

#include "jqcd.h"
#include "solver.h"

namespace jqcd {

struct Server;

Server *serve_create(int device, int sm_count, int hp, size_t budget, int max_slots, int max_queue,
                     std::string *err);
jqcd_status serve_submit(Server *S, GaugeEntry *G, const jqcd_request &r, uint64_t *ticket);
// PENDING while the request is queued or running; otherwise its final status
// (the ticket is forgotten when `forget`).
jqcd_status serve_poll(Server *S, uint64_t ticket, jqcd_solve_info *info, bool forget);
bool serve_uses_gauge(Server *S, const GaugeEntry *G);
// Waits until every submitted request has finished, then stops the thread.
jqcd_status serve_destroy(Server *S, jqcd_serve_stats *stats, std::string *err);

}  // namespace jqcd
