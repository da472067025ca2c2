"""FP64 CPU oracle of the coupled central-moment LB step (test infrastructure
only: imported by the tests, the smoke check and the benchmark's CPU-baseline
leg, never by the product package)."""
