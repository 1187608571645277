"""CPU oracle of the torchmSAT objective.  Test infrastructure only: imported
by the tests, the smoke check and the benchmark's CPU baseline, never by the
GPU library."""
