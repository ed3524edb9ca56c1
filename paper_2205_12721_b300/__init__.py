"""B300-native TMOP partial-assembly Newton step (package root; filled in below)."""
