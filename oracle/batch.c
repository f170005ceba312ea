/*
 * CPU oracle batch driver -- TEST INFRASTRUCTURE (tests/, __graft_entry__.smoke(), bench.py CPU baseline only).
 * Runs route A or route R over n quartics on a plain pthread pool; each quartic is independent.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

int qfs_oracle_height_a(int p, const uint8_t *f35, int max_h, int lift_signed, int32_t *g_out, int32_t *D_out,
                        int32_t *delta_out, int32_t *iters_out);
int qfs_oracle_height_r(int p, const uint8_t *f35, int max_h, int32_t *d1f_out, int32_t *iters_out);

typedef struct {
  int route, p, max_h;
  int64_t n;
  const uint8_t *coeffs;
  int8_t *out;
  int64_t next;
  pthread_mutex_t lock;
} job_t;

static void *worker(void *arg) {
  job_t *J = (job_t *)arg;
  for (;;) {
    pthread_mutex_lock(&J->lock);
    int64_t i = J->next++;
    pthread_mutex_unlock(&J->lock);
    if (i >= J->n) break;
    const uint8_t *f = J->coeffs + 35 * i;
    int h = J->route == 0 ? qfs_oracle_height_a(J->p, f, J->max_h, 0, 0, 0, 0, 0)
                          : qfs_oracle_height_r(J->p, f, J->max_h, 0, 0);
    J->out[i] = (int8_t)(h < -1 ? -2 : h);
  }
  return 0;
}

/* route: 0 = A (literal), 1 = R.  out[i] = height code; -2 marks an internal failure of the oracle. */
int qfs_oracle_heights(int route, int p, int64_t n, const uint8_t *coeffs, int max_h, int8_t *out, int threads) {
  if (n <= 0) return 0;
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  job_t J;
  J.route = route; J.p = p; J.max_h = max_h; J.n = n; J.coeffs = coeffs; J.out = out; J.next = 0;
  pthread_mutex_init(&J.lock, 0);
  pthread_t tid[256];
  int started = 0;
  for (int t = 0; t < threads; t++)
    if (pthread_create(&tid[t], 0, worker, &J) == 0) started++;
    else break;
  if (started == 0) worker(&J);
  for (int t = 0; t < started; t++) pthread_join(tid[t], 0);
  pthread_mutex_destroy(&J.lock);
  return 0;
}
