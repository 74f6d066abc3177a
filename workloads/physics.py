"""Physical constants used to generate trajectories (SI, CODATA 2018)."""
C0 = 299792458.0
Q_E = 1.602176634e-19
M_E = 9.1093837015e-31
EPS0 = 8.8541878128e-12
