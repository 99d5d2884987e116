/* Compiled as C99 against include/esd.h and linked with libesd.so: the boundary is a
 * plain C ABI.  Calls only entry points that need no GPU (host reference tables,
 * status strings, the host-side layout audit, argument rejection) and prints what it
 * read, one "key value" pair per line. */
#include <stdio.h>
#include <string.h>

#include "esd.h"
#include "esd_test.h"

int main(void) {
  esd_info info;
  memset(&info, 0, sizeof info);
  if (esd_ref_info(3, 4, &info) != ESD_OK) {
    fprintf(stderr, "esd_ref_info failed: %s\n", esd_last_error());
    return 1;
  }
  printf("n_modes %d\n", info.n_modes);
  printf("n_vol_nodes %d\n", info.n_vol_nodes);
  printf("n_facet_nodes %d\n", info.n_facet_nodes);
  printf("vol_pairs %lld\n", (long long)info.vol_pairs_per_elem);
  printf("facet_pairs %lld\n", (long long)info.facet_pairs_per_elem);
  printf("paper_flux_count %lld\n", (long long)info.paper_flux_count_per_elem);
  printf("unsupported_degree %d\n", (int)esd_ref_info(3, 11, &info));
  printf("null_output %d\n", (int)esd_ref_info(2, 4, NULL));
  printf("null_mesh_rhs %d\n", (int)esd_rhs(NULL, NULL, NULL, NULL));
  printf("layouts %d\n", (int)esd_debug_check_layouts());
  printf("status_string %s\n", esd_status_string(ESD_ERR_STATE));
  return 0;
}
