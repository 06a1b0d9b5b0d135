/* The C ABI from plain C99: the header compiles as C, the library links, and the
 * entry points that need no GPU validate their arguments.  Built and run by
 * tests/test_abi_host.py. */
#include <stdio.h>
#include <string.h>

#include "nbldpc.h"

#define CHECK(cond)                                              \
  do {                                                           \
    if (!(cond)) {                                               \
      fprintf(stderr, "failed: %s (line %d)\n", #cond, __LINE__); \
      return 1;                                                  \
    }                                                            \
  } while (0)

int main(void) {
  nbldpc_code *code = (nbldpc_code *)0x1;
  const int32_t row_ptr[2] = {0, 2}, col_idx[2] = {0, 1};
  const uint8_t coef[2] = {1, 1};
  size_t bytes = 0;
  int n_done = 0;
  nbldpc_server *srv = NULL;
  nbldpc_server_stats st;
  nbldpc_request req;

  CHECK(strcmp(nbldpc_status_string(NBLDPC_OK), "ok") == 0);
  CHECK(nbldpc_status_string(12345) != NULL);
  /* field order 3 is not a power of two: rejected before any device call */
  CHECK(nbldpc_code_create(3, 0x7, 2, 1, row_ptr, col_idx, coef, &code) == NBLDPC_ERR_POLY);
  CHECK(code == NULL);
  CHECK(nbldpc_code_create(4, 0x7, 2, 1, NULL, col_idx, coef, &code) == NBLDPC_ERR_ARG);
  CHECK(nbldpc_decode_workspace_size(NULL, 4, &bytes) == NBLDPC_ERR_ARG);
  CHECK(nbldpc_fftspa_workspace_size(NULL, 4, &bytes) == NBLDPC_ERR_ARG);
  CHECK(nbldpc_code_set_message_bits(NULL, 16) == NBLDPC_ERR_ARG);
  CHECK(nbldpc_code_set_cnp_schedule(NULL, NBLDPC_CNP_TABLE1) == NBLDPC_ERR_ARG);
  CHECK(nbldpc_server_create_custom(NULL, 1024, 1, 1, 0, &srv) == NBLDPC_ERR_ARG);
  CHECK(nbldpc_server_poll(NULL, NULL, 0, &n_done) == NBLDPC_ERR_ARG);
  CHECK(nbldpc_server_stats_get(NULL, &st) == NBLDPC_ERR_ARG);
  memset(&req, 0, sizeof req);
  CHECK(nbldpc_server_submit(NULL, &req, NULL) == NBLDPC_ERR_ARG);
  nbldpc_server_destroy(NULL);
  nbldpc_code_destroy(NULL);
  CHECK(NBLDPC_MAX_BATCH_JOBS == 32);
  printf("c99 abi ok\n");
  return 0;
}
