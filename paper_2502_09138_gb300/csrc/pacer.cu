// Publishing-rate control of an offline source (host-side).
//
// Section 3 of the paper: publishing as fast as possible and throttling the
// source only by the number of collisions in flight makes work arrive in
// waves; when a wave hits a slower serial stage the other stages run dry.
// ALICE instead smooths the publishing rate with a heuristic that keeps
// shortening the delay between publications, slowly, to put more collisions
// in flight, until back pressure appears.  The paper gives the behaviour,
// not the constants; the reading implemented here:
//   NAIVE   publish whenever fewer than max_in_flight frames are in flight
//           (published and not yet consumed).
//   SMOOTH  publish when fewer than max_in_flight are in flight AND the
//           publishing delay has passed since the last publication.  After
//           every consumed frame the delay shrinks by the factor
//           (1 - decrease) if no back pressure was seen since the previous
//           consumed frame, and grows by (1 + increase) otherwise; back
//           pressure = a publication attempt found the in-flight limit
//           reached or frames waiting for admission downstream (backlog).
//           The delay stays within [min_delay_s, max_delay_s].
// The pacer holds no clock and no thread: the caller passes its own time, so
// the same object drives a real source or a simulation.
#include <algorithm>
#include <new>

#include "tpct.h"

struct tpct_pacer {
  tpct_pacer_config cfg;
  double delay = 0.0;
  double last_publish = -1e300;
  bool pressure = false;
  int64_t published = 0, consumed = 0, pressure_events = 0;
};

extern "C" {

void tpct_default_pacer_config(tpct_pacer_config* c) {
  if (!c) return;
  c->policy = TPCT_PUBLISH_SMOOTH;
  c->max_in_flight = 8;
  c->initial_delay_s = 0.05;
  c->decrease = 0.02;
  c->increase = 0.05;
  c->min_delay_s = 0.0;
  c->max_delay_s = 10.0;
}

tpct_status tpct_pacer_create(const tpct_pacer_config* c, tpct_pacer** out) {
  if (!c || !out || c->max_in_flight < 1 || !(c->decrease >= 0.0 && c->decrease < 1.0) || !(c->increase >= 0.0) ||
      !(c->min_delay_s >= 0.0) || !(c->max_delay_s >= c->min_delay_s) ||
      (c->policy != TPCT_PUBLISH_NAIVE && c->policy != TPCT_PUBLISH_SMOOTH))
    return TPCT_E_INVALID;
  tpct_pacer* p = new (std::nothrow) tpct_pacer();
  if (!p) return TPCT_E_NOMEM;
  p->cfg = *c;
  p->delay = std::min(std::max(c->initial_delay_s, c->min_delay_s), c->max_delay_s);
  *out = p;
  return TPCT_OK;
}

void tpct_pacer_destroy(tpct_pacer* p) { delete p; }

int tpct_pacer_try_publish(tpct_pacer* p, double now_s, int32_t in_flight, int32_t backlog, double* wait_s) {
  if (!p) return 0;
  if (wait_s) *wait_s = 0.0;
  const bool smooth = p->cfg.policy == TPCT_PUBLISH_SMOOTH;
  if (in_flight >= p->cfg.max_in_flight || (smooth && backlog > 0)) {
    if (!p->pressure) ++p->pressure_events;
    p->pressure = true;
    return 0;   // wait for a consumed frame
  }
  if (smooth) {
    const double ready = p->last_publish + p->delay;
    if (now_s < ready) {
      if (wait_s) *wait_s = ready - now_s;
      return 0;
    }
  }
  p->last_publish = now_s;
  ++p->published;
  return 1;
}

void tpct_pacer_on_consumed(tpct_pacer* p, double now_s, int32_t in_flight, int32_t backlog) {
  (void)now_s;
  (void)in_flight;
  if (!p) return;
  ++p->consumed;
  if (p->cfg.policy != TPCT_PUBLISH_SMOOTH) return;
  if (p->pressure || backlog > 0)
    p->delay = std::min(p->cfg.max_delay_s, std::max(p->delay, 1e-6) * (1.0 + p->cfg.increase));
  else
    p->delay = std::max(p->cfg.min_delay_s, p->delay * (1.0 - p->cfg.decrease));
  p->pressure = false;
}

double tpct_pacer_delay(const tpct_pacer* p) { return p ? p->delay : 0.0; }

int64_t tpct_pacer_pressure_events(const tpct_pacer* p) { return p ? p->pressure_events : 0; }

}  // extern "C"
